"""GB300-native matrix-free modal DG + p-multigrid FGMRES implicit step.

The compute path is the CUDA library ``libdgpmg.so`` (sources under ``csrc/``)
behind the C ABI declared in ``include/dg.h``; ``binding`` marshals arguments
to it.  Importing this package loads nothing; the first call into
``binding`` loads the library and raises if it is missing.
"""
