// dg_residual_noalloc: the DG residual without any device allocation.
//
// Some callers cannot let a library call cudaMalloc at the moment they need a
// result: a solver embedded in a host application that reserved all device
// memory up front, or a time-critical loop that must not enter the CUDA
// allocator (it may synchronise the device or take a global lock).  This entry
// point serves them.  It computes exactly what dg_residual computes, with the
// same face kernel and the direct volume kernel, but the face-slot scratch lives in one file-scope device array of
// fixed size instead of in the mesh handle.  The array belongs to this file's
// device module, which the CUDA runtime may load lazily (on first use):
// dg_mesh_create looks the array up on its device, so the module and the
// array are in place before any mesh handle exists, and a call here finds
// them without any allocation.
//
// Limits and rules:
//  - the scratch holds NOALLOC_MAX_SLOTS doubles (8 MiB); a mesh needing more
//    (E * d * 2 * m * n_m doubles) is rejected with DG_ERR_INVALID;
//  - every GPU that loads the library reserves that array until the process exits;
//  - dg_mesh_create looks up the array's device address (cudaGetSymbolAddress)
//    on its current device, once per device; a device whose first mesh handle
//    cannot load the array fails there with DG_ERR_OOM, not here;
//  - on 3-D meshes and on Q_p meshes dg_residual evaluates the volume term by
//    sum factorisation and this entry point by the direct contractions: the
//    two results agree to rounding, not bit for bit;
//  - all calls share the array: calls that can overlap on the GPU (different
//    streams without ordering between them) race; order them on one stream;
//  - the array keeps the last call's contents; no part of it needs to start
//    at zero, because every slot read is first written by the same call.
#include <mutex>

#include "dg_internal.h"

namespace {

constexpr size_t NOALLOC_MAX_SLOTS = size_t(1) << 20;   // doubles (8 MiB)
static __device__ __align__(256) double g_noalloc_slots[NOALLOC_MAX_SLOTS];

constexpr int MAX_DEVICES = 64;
std::mutex g_lock;
double* g_addr[MAX_DEVICES] = {};

// Device address of the array on the current device (looked up once per device).
dg_status slots_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return DG_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_addr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_slots);
    if (e == cudaErrorMemoryAllocation) return DG_ERR_OOM;
    if (e != cudaSuccess || !p) return DG_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DG_OK;
}

}  // namespace

namespace dgk {
// Called by dg_mesh_create on the handle's device: loads the array (and the
// module that holds it) while allocation is still allowed.
dg_status noalloc_prepare() {
  double* p = nullptr;
  return slots_address(&p);
}
}  // namespace dgk

extern "C" dg_status dg_residual_noalloc(dg_mesh mesh, const double* W, const double* S, double* R,
                                         void* stream) {
  if (!mesh || !W || !R || R == W || (S && S == R)) return DG_ERR_INVALID;
  const dgk::Mesh& M = mesh->m;
  if (M.kind != dgk::DG_MESH_STRUCTURED) return DG_ERR_INVALID;
  const size_t need = (size_t)M.E * M.d * 2 * M.nb;
  if (need > NOALLOC_MAX_SLOTS) return DG_ERR_INVALID;
  double* slots = nullptr;
  dg_status s = slots_address(&slots);
  if (s != DG_OK) return s;
  const cudaError_t e = dgk::launch_residual_with_slots(M, W, S, R, slots, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) return DG_ERR_OOM;
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
