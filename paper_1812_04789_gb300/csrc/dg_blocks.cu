// Element Jacobian blocks, subspace inheritance and block Jacobi
// (Sec. 5.1 eq. ODEDG; Sec. 6.1 inheritance; Sec. 6.3 element block Jacobi).
//
// probe_kernel: one CTA per element (grid-stride).  The diagonal block
//   D_e[(v,i'),(w,i)] = dR_{e,v,i'}/dW_{e,w,i} + sigma |J| delta
// is a sum over the element's volume points and the points of its own faces of
//   Test_c(p, i') * J_p[(v,c),(w,s)] * Trial_s(p, i),
// where J_p is the pointwise derivative of the point outputs c (volume: the flux
// tensor F[v][k]; face: the numerical flux, the two lifting integrands and the
// dual-consistency tensor) with respect to the point inputs s of variable w
// (the value and the d gradient components), Trial_s is the basis value or
// gradient, and Test_c the matching test function (the BR2 lifting is linear,
// so it is folded into precomputed lifted test functions).  For each w the
// kernel takes chunks of points: (J) 1+d dual-number evaluations per point,
// (Y) Y = J . Trial, (G) a register-tiled accumulation of Test . Y into the
// block in global memory (each CTA owns its element's blocks: no atomics).
// Neighbour blocks dR_e/dW_nbr (first nmc modes only, Sec. 6.3: coarse order)
// use the same machinery with the seed on the neighbour's trace.  A direction
// with one element makes the element its own neighbour: the neighbour-side
// seed of such a face then adds to the diagonal block.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include <cuda_bf16.h>

#include "dg_internal.h"
#include "dg_probe.cuh"

namespace dgk {

constexpr int PROBE_QC = 8;    // points per contraction sub-chunk
constexpr int PROBE_CH = 8;    // columns per register tile
template <class T> struct ProbeJQC { static constexpr int value = 64; };   // points per Jacobian chunk
template <> struct ProbeJQC<double> { static constexpr int value = 32; };
constexpr int PROBE_RI = 4;    // test rows per register tile

__host__ __device__ inline size_t probe_align4(size_t x) { return (x + 3) & ~size_t(3); }
__host__ __device__ inline int probe_pad(int n) { return (n + PROBE_CH - 1) / PROBE_CH * PROBE_CH; }

// Per-CTA cache layout (elements of T; every buffer starts on a multiple of 4
// elements, so 16-byte vector loads of the tiles are aligned)
template <class T>
struct ProbeLayout {
  size_t cW, cU, cFU, Jb, Yb, Tb, total;
  __host__ __device__ ProbeLayout(int D, int nb, int nm, int nq, int nqf) {
    const int M = D + 2, nf = 2 * D, KM = 3 + D, nmp = probe_pad(nm);
    size_t o = 0;
    cW = o;  o = probe_align4(o + (size_t)(1 + nf) * nb);
    cU = o;  o = probe_align4(o + (size_t)nq * M * (1 + D));
    cFU = o; o = probe_align4(o + (size_t)nf * 2 * nqf * M * (1 + D));
    Jb = o;  o = probe_align4(o + (size_t)ProbeJQC<T>::value * (1 + D) * M * KM);
    Yb = o;  o = probe_align4(o + (size_t)PROBE_QC * M * KM * nmp);
    Tb = o;  o = probe_align4(o + (size_t)PROBE_QC * KM * nmp);
    total = o;
  }
};

enum ProbeTask : int { TASK_VOL = 0, TASK_FACE_OWN = 1, TASK_FACE_NBR = 2 };

template <class T>
struct ProbeCtx {
  MeshView<T> mv;
  Phys<T> ph;
  T half_eta;
  const T* cU;
  const T* cFU;
  T* Jb;
  T* Yb;
  T* Tb;
};

// 16-byte vector loads of N consecutive elements (aligned by construction)
template <int N>
__device__ __forceinline__ void vload(const float* p, float* out) {
#pragma unroll
  for (int j = 0; j < N; j += 4) {
    float4 x = *reinterpret_cast<const float4*>(p + j);
    out[j] = x.x; out[j + 1] = x.y; out[j + 2] = x.z; out[j + 3] = x.w;
  }
}
template <int N>
__device__ __forceinline__ void vload(const double* p, double* out) {
#pragma unroll
  for (int j = 0; j < N; j += 2) {
    double2 x = *reinterpret_cast<const double2*>(p + j);
    out[j] = x.x; out[j + 1] = x.y;
  }
}

// One sweep: points [0, npts) of a task, seed variable w, accumulated into the
// target block rows (v, i' < nmo) x columns (w, i < nmi), leading dimension ld.
template <int D, class T>
__device__ __forceinline__ void probe_sweep(const ProbeCtx<T>& cx, int task, int sface, int npts, int w, int nmo,
                                            int nmi, T* __restrict__ tgt, int ld) {
  constexpr int M = D + 2, KM = 3 + D, PU = M * (1 + D), NS = 1 + D;
  constexpr int JQC = ProbeJQC<T>::value;
  const MeshView<T>& mv = cx.mv;
  const int nm = mv.nm, nq = mv.nq, nqf = mv.nqf;
  const int nk = task == TASK_VOL ? D : KM;
  const int nmp = probe_pad(nmi);
  T* Jb = cx.Jb;
  T* Yb = cx.Yb;
  T* Tb = cx.Tb;
  for (int cj = 0; cj < npts; cj += JQC) {
    const int ncj = min(JQC, npts - cj);
    // (J) pointwise derivatives for the 1+d unit seeds of variable w
    for (int t = threadIdx.x; t < ncj * NS; t += blockDim.x) {
      const int pl = t / NS, sd = t % NS, pt = cj + pl;
      T* jo = Jb + ((size_t)pl * NS + sd) * M * KM;
      if (task == TASK_VOL) {
        using S = Dual<T>;
        const T* pu = cx.cU + (size_t)pt * PU;
        S u[M], g[M][D], F[M][D];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          u[v] = S(pu[v], (v == w && sd == 0) ? T(1) : T(0));
#pragma unroll
          for (int kk = 0; kk < D; ++kk) g[v][kk] = S(pu[M + v * D + kk], (v == w && sd == 1 + kk) ? T(1) : T(0));
        }
        flux_total<D, S, T>(u, g, F, cx.ph);
#pragma unroll
        for (int v = 0; v < M; ++v)
#pragma unroll
          for (int kk = 0; kk < D; ++kk) jo[v * KM + kk] = F[v][kk].d;
      } else {
        const int s = task == TASK_FACE_OWN ? pt / nqf : sface;
        const int q = task == TASK_FACE_OWN ? pt % nqf : pt;
        const bool own = task == TASK_FACE_OWN;
        T sgo[D], sgn[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) {
          sgo[kk] = (own && sd == 1 + kk) ? T(1) : T(0);
          sgn[kk] = (!own && sd == 1 + kk) ? T(1) : T(0);
        }
        T oGL[M], oGR[M], oFp[M], oDo[M * D];
        face_point_tangent<D, T>(cx.cFU + ((size_t)(s * 2) * nqf + q) * PU, cx.cFU + ((size_t)(s * 2 + 1) * nqf + q) * PU,
                                 s / 2, s % 2, w, (own && sd == 0) ? T(1) : T(0), sgo, (!own && sd == 0) ? T(1) : T(0),
                                 sgn, cx.ph, oGL, oGR, oFp, oDo);
#pragma unroll
        for (int v = 0; v < M; ++v) {
          jo[v * KM + 0] = oFp[v];
          jo[v * KM + 1] = oGL[v];
          jo[v * KM + 2] = oGR[v];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) jo[v * KM + 3 + kk] = oDo[v * D + kk];
        }
      }
    }
    __syncthreads();
    for (int c0 = cj; c0 < cj + ncj; c0 += PROBE_QC) {
      const int nc = min(PROBE_QC, cj + ncj - c0);
      // (Y) contraction with the trial functions of the seeded trace, and the
      // test functions of the sub-chunk's points (independent of v and w);
      // rows are padded to a multiple of PROBE_CH with zeros
      // one warp per (point, output kind) row; the lanes run over the modes and
      // produce Y for every variable v at once (the trial values are shared)
      const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
      for (int row = threadIdx.x >> 5; row < nc * nk; row += nwarp) {
        const int pl = row / nk, kind = row - pl * nk, pt = c0 + pl;
        T jv[M][NS];
#pragma unroll
        for (int v = 0; v < M; ++v)
#pragma unroll
          for (int sd = 0; sd < NS; ++sd) jv[v][sd] = Jb[((size_t)(pt - cj) * NS + sd) * M * KM + v * KM + kind];
        int f = 0, s = 0, q = pt;
        T tscale = T(0);
        const T* trow = nullptr;
        if (task == TASK_VOL) {
          tscale = -mv.vw[pt];
          trow = mv.vdphi + ((size_t)kind * nq + pt) * nm;
        } else {
          s = task == TASK_FACE_OWN ? pt / nqf : sface;
          q = task == TASK_FACE_OWN ? pt % nqf : pt;
          f = task == TASK_FACE_OWN ? s : (s ^ 1);
          // test functions live on the element's own face s
          const T sg = (s % 2) ? T(1) : T(-1);
          const T fwq = mv.fw[(size_t)(s / 2) * nqf + q];
          if (kind == 0) {
            tscale = sg * fwq;
            trow = mv.fphi + ((size_t)s * nqf + q) * nm;
          } else if (kind < 3) {
            tscale = sg * cx.half_eta;
            trow = mv.liftT + (((size_t)s * 2 + (kind - 1)) * nqf + q) * nm;
          } else {
            tscale = -fwq;
            trow = mv.fdphi + (((size_t)s * D + (kind - 3)) * nqf + q) * nm;
          }
        }
        for (int i = lane; i < nmp; i += 32) {
          T phi[NS];
          T test = T(0);
          if (i < nmi) {
            if (task == TASK_VOL) {
              phi[0] = mv.vphi[(size_t)pt * nm + i];
#pragma unroll
              for (int kk = 0; kk < D; ++kk) phi[1 + kk] = mv.vdphi[((size_t)kk * nq + pt) * nm + i];
            } else {
              phi[0] = mv.fphi[((size_t)f * nqf + q) * nm + i];
#pragma unroll
              for (int kk = 0; kk < D; ++kk) phi[1 + kk] = mv.fdphi[(((size_t)f * D + kk) * nqf + q) * nm + i];
            }
            test = tscale * trow[i];
          } else {
#pragma unroll
            for (int sd = 0; sd < NS; ++sd) phi[sd] = T(0);
          }
#pragma unroll
          for (int v = 0; v < M; ++v) {
            T y = T(0);
#pragma unroll
            for (int sd = 0; sd < NS; ++sd) y += jv[v][sd] * phi[sd];
            Yb[(((size_t)pl * M + v) * nk + kind) * nmp + i] = y;
          }
          Tb[((size_t)pl * nk + kind) * nmp + i] = test;
        }
      }
      __syncthreads();
      // (G) tgt[(v,i'),(w,i)] += sum_{points, kinds} Test(p, kind, i') Y[p][v][kind][i],
      // each thread a PROBE_RI x PROBE_CH register tile
      const int nch = nmp / PROBE_CH, nib = (nmo + PROBE_RI - 1) / PROBE_RI;
      for (int t = threadIdx.x; t < M * nib * nch; t += blockDim.x) {
        const int ch = t % nch, r = t / nch, ib = r % nib, v = r / nib;
        const int i0 = ch * PROBE_CH, ip0 = ib * PROBE_RI;
        T acc[PROBE_RI][PROBE_CH];
#pragma unroll
        for (int a = 0; a < PROBE_RI; ++a)
#pragma unroll
          for (int c = 0; c < PROBE_CH; ++c) acc[a][c] = T(0);
        for (int pl = 0; pl < nc; ++pl) {
          for (int kind = 0; kind < nk; ++kind) {
            T tv[PROBE_RI], yv[PROBE_CH];
            vload<PROBE_RI>(Tb + ((size_t)pl * nk + kind) * nmp + ip0, tv);
            vload<PROBE_CH>(Yb + (((size_t)pl * M + v) * nk + kind) * nmp + i0, yv);
#pragma unroll
            for (int a = 0; a < PROBE_RI; ++a)
#pragma unroll
              for (int c = 0; c < PROBE_CH; ++c) acc[a][c] += tv[a] * yv[c];
          }
        }
#pragma unroll
        for (int a = 0; a < PROBE_RI; ++a) {
          const int ip = ip0 + a;
          if (ip < nmo) {
            T* row = tgt + (size_t)(v * nmo + ip) * ld + (size_t)w * nmi + i0;
#pragma unroll
            for (int c = 0; c < PROBE_CH; ++c)
              if (i0 + c < nmi) row[c] += acc[a][c];
          }
        }
      }
      __syncthreads();
    }
  }
}

template <int D, class T>
__global__ void __launch_bounds__(256) probe_kernel(MeshView<T> mv, Phys<T> ph, const T* __restrict__ W,
                                                    T sigma, T* __restrict__ Dout, size_t dstride,
                                                    T* __restrict__ Oout, int nmc, T* gscratch, int use_smem,
                                                    int nbr_only, int* status) {
  constexpr int M = D + 2, NF = 2 * D, PU = M * (1 + D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, nqf = mv.nqf, E = mv.E;
  const ProbeLayout<T> L(D, nb, nm, nq, nqf);
  T* C = use_smem ? reinterpret_cast<T*>(smem_raw) : gscratch + (size_t)blockIdx.x * L.total;
  T* cW = C + L.cW;
  T* cU = C + L.cU;
  T* cFU = C + L.cFU;
  ProbeCtx<T> cx;
  cx.mv = mv;
  cx.ph = ph;
  cx.half_eta = T(0.5) * ph.eta;
  cx.cU = cU;
  cx.cFU = cFU;
  cx.Jb = C + L.Jb;
  cx.Yb = C + L.Yb;
  cx.Tb = C + L.Tb;
  const int nbc = M * nmc;
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    int nbrs[NF];
#pragma unroll
    for (int s = 0; s < NF; ++s) nbrs[s] = mv.nbr[e * NF + s];
    T* De = Dout + (size_t)e * dstride;
    if (!nbr_only)
      for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) De[t] = (t / nb == t % nb) ? sigma * mv.detJ : T(0);
    if (Oout)
      for (int t = threadIdx.x; t < NF * nbc * nbc; t += blockDim.x) Oout[(size_t)e * NF * nbc * nbc + t] = T(0);
    probe_stage_primal<D, T>(mv, ph, W, e, nbrs, cW, cU, cFU, !nbr_only, status);
    for (int w = 0; w < M; ++w) {
      if (!nbr_only) {
        probe_sweep<D, T>(cx, TASK_VOL, -1, nq, w, nm, nm, De, nb);
        probe_sweep<D, T>(cx, TASK_FACE_OWN, -1, NF * nqf, w, nm, nm, De, nb);
      }
      for (int s = 0; s < NF; ++s) {
        if (nbrs[s] == e) {
          probe_sweep<D, T>(cx, TASK_FACE_NBR, s, nqf, w, nm, nm, De, nb);
        } else if (Oout != nullptr) {
          probe_sweep<D, T>(cx, TASK_FACE_NBR, s, nqf, w, nmc, nmc, Oout + ((size_t)e * NF + s) * nbc * nbc, nbc);
        }
      }
    }
    __syncthreads();
  }
}

template <class T>
size_t probe_scratch_elems(const Mesh& M, int nmc, bool* fits_smem) {
  (void)nmc;
  ProbeLayout<T> L(M.d, M.nb, M.nm, M.nq, M.nqf);
  size_t bytes = L.total * sizeof(T);
  *fits_smem = bytes <= 220 * 1024;
  return L.total;
}
template size_t probe_scratch_elems<double>(const Mesh&, int, bool*);
template size_t probe_scratch_elems<float>(const Mesh&, int, bool*);

static int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// grid used when the caches live in global scratch
int probe_grid_global() { return 2 * num_sms(); }

template <int D, class T>
static cudaError_t run_probe(const Mesh& Ms, const T* W, T sigma, T* Dout, size_t dstride, T* Oout, int nmc,
                             T* scratch, size_t scratch_elems, bool nbr_only, cudaStream_t st) {
  bool fits;
  size_t tot = probe_scratch_elems<T>(Ms, nmc, &fits);
  int grid;
  size_t smem = 0;
  if (fits) {
    smem = tot * sizeof(T);
    grid = Ms.E;
    if (smem > 48 * 1024)
      allow_max_smem(probe_kernel<D, T>);
  } else {
    grid = std::min(Ms.E, probe_grid_global());
    if (!scratch || scratch_elems < tot * (size_t)grid) return cudaErrorInvalidValue;
  }
  note_launch();
  probe_kernel<D, T><<<grid, 256, smem, st>>>(Ms.view<T>(), Ms.phys_t<T>(), W, sigma, Dout, dstride, Oout,
                                             nmc, scratch, fits ? 1 : 0, nbr_only ? 1 : 0, Ms.status);
  return cudaGetLastError();
}

// FP32 blocks go through the tensor-core kernel when the mesh has a plan for
// it (DG_PROBE_SIMT=1 in the environment selects the SIMT kernel instead); the
// coarse neighbour blocks then come from probe_nbr_kernel, or, when a
// direction has one element (its faces feed the diagonal block), from the SIMT
// kernel restricted to the neighbour-seeded terms.
static bool use_tc(const Mesh& M) {
  const char* e = getenv("DG_PROBE_SIMT");
  return M.tc.ok && M.tc_test && M.tc_trial && !(e && e[0] == '1');
}

template <class T>
cudaError_t launch_probe_blocks(const Mesh& M, const T* W, T sigma, T* D, size_t dstride, T* O, int nmc,
                                int nbr_colmajor, T* scratch, size_t scratch_elems, cudaStream_t st) {
  if (std::is_same<T, float>::value && nbr_colmajor && O) {
    // layout fixed at setup: the neighbour blocks always come from probe_nbr_kernel
    cudaError_t e = use_tc(M) ? launch_probe_tc(M, (const float*)W, (float)sigma, (float*)D, dstride, st)
                   : M.d == 2 ? run_probe<2, T>(M, W, sigma, D, dstride, nullptr, 0, scratch, scratch_elems, false, st)
                              : run_probe<3, T>(M, W, sigma, D, dstride, nullptr, 0, scratch, scratch_elems, false, st);
    if (e != cudaSuccess) return e;
    return launch_probe_nbr(M, (const float*)W, (float*)O, nmc, 1, st);
  }
  bool nbr_only = false;
  if (std::is_same<T, float>::value && use_tc(M)) {
    cudaError_t e = launch_probe_tc(M, (const float*)W, (float)sigma, (float*)D, dstride, st);
    if (e != cudaSuccess) return e;
    bool self = false;
    for (int k = 0; k < M.d; ++k) self = self || M.desc.n[k] == 1;
    if (O == nullptr && !self) return cudaSuccess;
    if (!self && probe_nbr_fits(M, nmc)) return launch_probe_nbr(M, (const float*)W, (float*)O, nmc, 0, st);
    nbr_only = true;
  }
  if (M.d == 2) return run_probe<2, T>(M, W, sigma, D, dstride, O, nmc, scratch, scratch_elems, nbr_only, st);
  return run_probe<3, T>(M, W, sigma, D, dstride, O, nmc, scratch, scratch_elems, nbr_only, st);
}
template cudaError_t launch_probe_blocks<double>(const Mesh&, const double*, double, double*, size_t, double*,
                                                 int, int, double*, size_t, cudaStream_t);
template cudaError_t launch_probe_blocks<float>(const Mesh&, const float*, float, float*, size_t, float*, int,
                                                int, float*, size_t, cudaStream_t);

bool probe_nbr_colmajor_ok(const Mesh& M, int nmc) { return use_tc(M) && probe_nbr_fits(M, nmc); }

// ---------------------------------------------------------------- truncation
template <class T>
__global__ void truncate_kernel(const T* __restrict__ src, int nms, size_t sstride, int src_t, T* __restrict__ dst,
                                int nmt, size_t dstride, int dst_t, int m, long nblk) {
  const int nbs = m * nms, nbt = m * nmt, lds = inv_ld<T>(nbs), ldt = inv_ld<T>(nbt);
  const long tot = nblk * nbt * nbt;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    const long b = t / ((long)nbt * nbt);
    const int r = (int)(t % ((long)nbt * nbt));
    // consecutive t walk the destination's contiguous dimension
    const int a1 = r / nbt, a2 = r % nbt;
    const int row = dst_t ? a2 : a1, col = dst_t ? a1 : a2;
    const int v = row / nmt, i = row % nmt, w = col / nmt, j = col % nmt;
    const int rs = v * nms + i, cs = w * nms + j;
    const T x = src[(size_t)b * sstride + (src_t ? (size_t)cs * lds + rs : (size_t)rs * nbs + cs)];
    dst[(size_t)b * dstride + (dst_t ? (size_t)col * ldt + row : (size_t)row * nbt + col)] = x;
  }
}

template <class T>
cudaError_t launch_truncate_blocks(const T* src, int nms, size_t sstride, int src_t, T* dst, int nmt,
                                   size_t dstride, int dst_t, int m, long nblk, cudaStream_t st) {
  long tot = nblk * (long)(m * nmt) * (m * nmt);
  if (tot <= 0) return cudaSuccess;
  long grid = std::min<long>((tot + 255) / 256, 65535L * 8);
  note_launch();
  truncate_kernel<T><<<(int)grid, 256, 0, st>>>(src, nms, sstride, src_t, dst, nmt, dstride, dst_t, m, nblk);
  return cudaGetLastError();
}
template cudaError_t launch_truncate_blocks<double>(const double*, int, size_t, int, double*, int, size_t, int, int,
                                                    long, cudaStream_t);
template cudaError_t launch_truncate_blocks<float>(const float*, int, size_t, int, float*, int, size_t, int, int,
                                                   long, cudaStream_t);

// ---------------------------------------------------------------- block apply / BSR
// One CTA per element: the element's input (and neighbours' for BSR) staged in
// shared memory; each warp takes two block rows at a time, the lanes striding
// the columns with an unrolled loop (coalesced row reads, several loads in
// flight per lane, conflict-free shared reads); fixed butterfly reductions.
template <class T>
__device__ __forceinline__ void row_dot2(const T* __restrict__ A0, const T* __restrict__ A1, const T* xs, int n,
                                         int lane, T& s0, T& s1) {
#pragma unroll 4
  for (int c = lane; c < n; c += 32) {
    const T xv = xs[c];
    s0 += __ldg(A0 + c) * xv;
    s1 += __ldg(A1 + c) * xv;
  }
}

template <class T>
__global__ void __launch_bounds__(256) bsr_kernel(const T* __restrict__ Dm, size_t dstride,
                                                  const T* __restrict__ O, const int* __restrict__ nbr, int nf,
                                                  const T* __restrict__ x, T* __restrict__ y, int nb, int E) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);   // [(1 + nf)][nb]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nsrc = O ? 1 + nf : 1;
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    for (int t = threadIdx.x; t < nsrc * nb; t += blockDim.x) {
      int who = t / nb, j = t % nb;
      int el = who == 0 ? e : nbr[(size_t)e * nf + who - 1];
      xs[t] = x[(size_t)el * nb + j];
    }
    __syncthreads();
    for (int r0 = 2 * warp; r0 < nb; r0 += 2 * nw) {
      const int r1 = min(r0 + 1, nb - 1);     // an odd last row is computed twice, stored once
      T s0 = T(0), s1 = T(0);
      row_dot2<T>(Dm + (size_t)e * dstride + (size_t)r0 * nb, Dm + (size_t)e * dstride + (size_t)r1 * nb, xs, nb,
                  lane, s0, s1);
      if (O) {
        for (int s = 0; s < nf; ++s) {
          const T* Ob = O + ((size_t)e * nf + s) * dstride;
          row_dot2<T>(Ob + (size_t)r0 * nb, Ob + (size_t)r1 * nb, xs + (size_t)(1 + s) * nb, nb, lane, s0, s1);
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
      }
      if (lane == 0) {
        y[(size_t)e * nb + r0] = s0;
        if (r1 != r0) y[(size_t)e * nb + r1] = s1;
      }
    }
    __syncthreads();
  }
}

// Block-Jacobi apply on column-major inverses (leading dimension ld = inv_ld(nb)):
// each thread owns 16 bytes of rows (4 FP32 or 2 FP64) of one element and
// streams the columns with one vector load each (read-only, not kept in L1:
// the blocks are read once per apply); `epc` elements per CTA pass share the
// staged inputs.  No reductions: every thread finishes its own rows.
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  static constexpr int N = 4;
  __device__ __forceinline__ static void load(const float* p, float* v) {
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "l"(p));
  }
};
template <>
struct Vec16<double> {
  static constexpr int N = 2;
  __device__ __forceinline__ static void load(const double* p, double* v) {
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p));
  }
};

template <class T>
__global__ void __launch_bounds__(256) bj_colmajor_kernel(const T* __restrict__ A, size_t bstride,
                                                          const T* __restrict__ x, T* __restrict__ y, int nb,
                                                          int ld, int E, int epc, int tpe) {
  constexpr int R = Vec16<T>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);   // [epc][nb]
  const int sub = threadIdx.x / tpe, tt = threadIdx.x - sub * tpe;
  for (long e0 = (long)blockIdx.x * epc; e0 < E; e0 += (long)gridDim.x * epc) {
    const int nl = (int)min((long)epc, E - e0);
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) xs[t] = x[(size_t)e0 * nb + t];
    __syncthreads();
    if (sub < nl) {
      const T* base = A + (size_t)(e0 + sub) * bstride + R * tt;
      const T* xe = xs + (size_t)sub * nb;
      T acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = T(0);
#pragma unroll 8
      for (int c = 0; c < nb; ++c) {
        T a[R];
        Vec16<T>::load(base + (size_t)c * ld, a);
        const T xv = xe[c];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += a[j] * xv;
      }
      T* yo = y + (size_t)(e0 + sub) * nb + R * tt;
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (R * tt + j < nb) yo[j] = acc[j];
    }
    __syncthreads();
  }
}

template <class T>
cudaError_t launch_block_apply(const T* A, size_t bstride, int transposed, const T* r, T* z, int nb, int E,
                               cudaStream_t st) {
  if (transposed) {
    const int ld = inv_ld<T>(nb), tpe = ld / Vec16<T>::N;
    const int epc = std::max(1, 256 / tpe);
    const int threads = (epc * tpe + 31) / 32 * 32;
    const int grid = std::min((E + epc - 1) / epc, 8 * num_sms());
    note_launch();
    bj_colmajor_kernel<T><<<grid, threads, (size_t)epc * nb * sizeof(T), st>>>(A, bstride, r, z, nb, ld, E, epc,
                                                                                tpe);
    return cudaGetLastError();
  }
  int grid = std::min(E, 32 * num_sms());
  note_launch();
  bsr_kernel<T><<<grid, 256, nb * sizeof(T), st>>>(A, bstride, nullptr, nullptr, 0, r, z, nb, E);
  return cudaGetLastError();
}
template cudaError_t launch_block_apply<double>(const double*, size_t, int, const double*, double*, int, int,
                                                cudaStream_t);
template cudaError_t launch_block_apply<float>(const float*, size_t, int, const float*, float*, int, int,
                                               cudaStream_t);

template <class T>
__global__ void unpack_inverse_kernel(const T* __restrict__ A, size_t bstride, int transposed, T* __restrict__ out,
                                      int nb, int ld, long nblk) {
  const long tot = nblk * nb * nb;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    const long b = t / ((long)nb * nb);
    const int rc = (int)(t - b * nb * nb), r = rc / nb, c = rc - r * nb;
    out[t] = A[(size_t)b * bstride + (transposed ? (size_t)c * ld + r : (size_t)r * nb + c)];
  }
}

template <class T>
cudaError_t launch_unpack_inverse(const T* A, size_t bstride, int transposed, T* out, int nb, long nblk,
                                  cudaStream_t st) {
  const long tot = nblk * (long)nb * nb;
  if (tot <= 0) return cudaSuccess;
  note_launch();
  unpack_inverse_kernel<T><<<(int)std::min<long>((tot + 255) / 256, 65535L * 8), 256, 0, st>>>(
      A, bstride, transposed, out, nb, inv_ld<T>(nb), nblk);
  return cudaGetLastError();
}
template cudaError_t launch_unpack_inverse<double>(const double*, size_t, int, double*, int, long, cudaStream_t);
template cudaError_t launch_unpack_inverse<float>(const float*, size_t, int, float*, int, long, cudaStream_t);

// Block-sparse mat-vec on column-major blocks (leading dimension ld =
// inv_ld(nb)): y_e = D_e x_e + sum_s O_{e,s} x_nbr(e,s).  A thread owns one
// block b of one element and 16 bytes of its rows and streams the block's
// columns with one vector load each (so an element keeps (1 + 2d) ld / 4 FP32
// threads busy); the element's and its neighbours' inputs are staged in shared
// memory and the per-block partial rows are summed in a fixed order.
template <class T>
__global__ void __launch_bounds__(256) bsr_colmajor_kernel(const T* __restrict__ Dm, const T* __restrict__ O,
                                                           size_t bstride, const int* __restrict__ nbr, int nf,
                                                           const T* __restrict__ x, T* __restrict__ y, int nb,
                                                           int ld, int E, int epc, int tpe) {
  constexpr int R = Vec16<T>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nsrc = 1 + nf, tpb = nsrc * tpe;
  T* xs = reinterpret_cast<T*>(smem_raw);           // [epc][nsrc][nb]
  T* part = xs + (size_t)epc * nsrc * nb;           // [epc][nsrc][ld]
  const int sub = threadIdx.x / tpb, r = threadIdx.x - sub * tpb, b = r / tpe, tt = r - b * tpe;
  for (long e0 = (long)blockIdx.x * epc; e0 < E; e0 += (long)gridDim.x * epc) {
    const int nl = (int)min((long)epc, E - e0);
    for (int t = threadIdx.x; t < nl * nsrc * nb; t += blockDim.x) {
      const int el = t / (nsrc * nb), q = t - el * nsrc * nb, who = q / nb, j = q - who * nb;
      const long e = e0 + el;
      const long src = who == 0 ? e : nbr[(size_t)e * nf + who - 1];
      xs[t] = x[(size_t)src * nb + j];
    }
    __syncthreads();
    if (sub < nl) {
      const long e = e0 + sub;
      const T* base = (b == 0 ? Dm + (size_t)e * bstride : O + ((size_t)e * nf + b - 1) * bstride) + R * tt;
      const T* xb = xs + ((size_t)sub * nsrc + b) * nb;
      T acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = T(0);
#pragma unroll 8
      for (int c = 0; c < nb; ++c) {
        T a[R];
        Vec16<T>::load(base + (size_t)c * ld, a);
        const T xv = xb[c];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += a[j] * xv;
      }
      T* pr = part + ((size_t)sub * nsrc + b) * ld + R * tt;
#pragma unroll
      for (int j = 0; j < R; ++j) pr[j] = acc[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
      const int el = t / nb, row = t - el * nb;
      const T* pe = part + (size_t)el * nsrc * ld + row;
      T sum = T(0);
      for (int bb = 0; bb < nsrc; ++bb) sum += pe[(size_t)bb * ld];
      y[(size_t)(e0 + el) * nb + row] = sum;
    }
    __syncthreads();
  }
}

template <class T>
cudaError_t launch_bsr(const T* D, const T* O, size_t bstride, int transposed, const int* nbr, int nf, const T* x,
                       T* y, int nb, int E, cudaStream_t st) {
  if (transposed) {
    const int ld = inv_ld<T>(nb), tpe = ld / Vec16<T>::N, tpb = (1 + nf) * tpe;
    if (tpb <= 256) {
      const int epc = std::max(1, 256 / tpb);
      const int threads = (epc * tpb + 31) / 32 * 32;
      const int grid = std::min((E + epc - 1) / epc, 16 * num_sms());
      const size_t smem = (size_t)epc * (1 + nf) * (nb + ld) * sizeof(T);
      note_launch();
      bsr_colmajor_kernel<T><<<grid, threads, smem, st>>>(D, O, bstride, nbr, nf, x, y, nb, ld, E, epc, tpe);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;   // coarse blocks this large are stored row-major
  }
  int grid = std::min(E, 32 * num_sms());
  size_t smem = (size_t)(1 + nf) * nb * sizeof(T);
  note_launch();
  bsr_kernel<T><<<grid, 256, smem, st>>>(D, bstride, O, nbr, nf, x, y, nb, E);
  return cudaGetLastError();
}
template cudaError_t launch_bsr<double>(const double*, const double*, size_t, int, const int*, int, const double*,
                                        double*, int, int, cudaStream_t);
template cudaError_t launch_bsr<float>(const float*, const float*, size_t, int, const int*, int, const float*,
                                       float*, int, int, cudaStream_t);


// ---------------------------------------------------------------- BF16 block storage
// Blocks kept in BF16 for the mixed-precision smoothers (the workload's BF16
// preconditioner storage): column-major with leading dimension ld16 = nb
// rounded up to 8 (16 bytes), padding rows zero; products and sums in FP32.
// A thread owns 8 rows of one block and streams its columns with one 16-byte
// load each (8 BF16 values, widened by a shift), exactly like the FP32
// column-major kernels with twice the rows per load.
__global__ void to_bf16_kernel(const float* __restrict__ src, size_t sstride, int src_t, int ld_src,
                               unsigned short* __restrict__ dst, size_t dstride, int ld16, int nb, long nblk) {
  const long tot = nblk * (long)nb * ld16;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    const long b = t / ((long)nb * ld16);
    const int q = (int)(t - b * (long)nb * ld16), c = q / ld16, r = q - c * ld16;
    float v = 0.f;
    if (r < nb) v = src[(size_t)b * sstride + (src_t ? (size_t)c * ld_src + r : (size_t)r * nb + c)];
    dst[(size_t)b * dstride + (size_t)c * ld16 + r] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
}

cudaError_t launch_to_bf16(const float* src, size_t sstride, int src_t, unsigned short* dst, int nb, long nblk,
                           cudaStream_t st) {
  const long tot = nblk * (long)nb * ld_bf16(nb);
  if (tot <= 0) return cudaSuccess;
  note_launch();
  to_bf16_kernel<<<(int)std::min<long>((tot + 255) / 256, 65535L * 8), 256, 0, st>>>(
      src, sstride, src_t, inv_ld<float>(nb), dst, (size_t)nb * ld_bf16(nb), ld_bf16(nb), nb, nblk);
  return cudaGetLastError();
}

__global__ void unpack_bf16_kernel(const unsigned short* __restrict__ A, float* __restrict__ out, int nb, int ld16,
                                   long nblk) {
  const long tot = nblk * nb * nb;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    const long b = t / ((long)nb * nb);
    const int rc = (int)(t - b * nb * nb), r = rc / nb, c = rc - r * nb;
    out[t] = __uint_as_float((unsigned)A[(size_t)b * nb * ld16 + (size_t)c * ld16 + r] << 16);
  }
}

cudaError_t launch_unpack_bf16(const unsigned short* A, float* out, int nb, long nblk, cudaStream_t st) {
  const long tot = nblk * (long)nb * nb;
  if (tot <= 0) return cudaSuccess;
  note_launch();
  unpack_bf16_kernel<<<(int)std::min<long>((tot + 255) / 256, 65535L * 8), 256, 0, st>>>(A, out, nb, ld_bf16(nb),
                                                                                      nblk);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) bj_bf16_kernel(const unsigned short* __restrict__ A,
                                                      const float* __restrict__ x, float* __restrict__ y, int nb,
                                                      int ld16, int E, int epc, int tpe) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* xs = reinterpret_cast<float*>(smem_raw);   // [epc][nb]
  const int sub = threadIdx.x / tpe, tt = threadIdx.x - sub * tpe;
  const size_t bstride = (size_t)nb * ld16;
  for (long e0 = (long)blockIdx.x * epc; e0 < E; e0 += (long)gridDim.x * epc) {
    const int nl = (int)min((long)epc, E - e0);
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) xs[t] = x[(size_t)e0 * nb + t];
    __syncthreads();
    if (sub < nl) {
      const unsigned short* base = A + (size_t)(e0 + sub) * bstride + 8 * tt;
      const float* xe = xs + (size_t)sub * nb;
      float acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll 8
      for (int c = 0; c < nb; ++c) {
        float a[8];
        ld_bf16x8(base + (size_t)c * ld16, a);
        const float xv = xe[c];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += a[j] * xv;
      }
      float* yo = y + (size_t)(e0 + sub) * nb + 8 * tt;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (8 * tt + j < nb) yo[j] = acc[j];
    }
    __syncthreads();
  }
}

cudaError_t launch_block_apply_bf16(const unsigned short* A, const float* r, float* z, int nb, int E,
                                    cudaStream_t st) {
  const int ld16 = ld_bf16(nb), tpe = ld16 / 8;
  if (tpe > 256) return cudaErrorInvalidValue;
  const int epc = std::max(1, 256 / tpe);
  const int threads = (epc * tpe + 31) / 32 * 32;
  const int grid = std::min((E + epc - 1) / epc, 8 * num_sms());
  note_launch();
  bj_bf16_kernel<<<grid, threads, (size_t)epc * nb * sizeof(float), st>>>(A, r, z, nb, ld16, E, epc, tpe);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) bsr_bf16_kernel(const unsigned short* __restrict__ Dm,
                                                       const unsigned short* __restrict__ O,
                                                       const int* __restrict__ nbr, int nf,
                                                       const float* __restrict__ x, float* __restrict__ y, int nb,
                                                       int ld16, int E, int epc, int tpe) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nsrc = 1 + nf, tpb = nsrc * tpe;
  const size_t bstride = (size_t)nb * ld16;
  float* xs = reinterpret_cast<float*>(smem_raw);   // [epc][nsrc][nb]
  float* part = xs + (size_t)epc * nsrc * nb;       // [epc][nsrc][ld16]
  const int sub = threadIdx.x / tpb, r = threadIdx.x - sub * tpb, b = r / tpe, tt = r - b * tpe;
  for (long e0 = (long)blockIdx.x * epc; e0 < E; e0 += (long)gridDim.x * epc) {
    const int nl = (int)min((long)epc, E - e0);
    for (int t = threadIdx.x; t < nl * nsrc * nb; t += blockDim.x) {
      const int el = t / (nsrc * nb), q = t - el * nsrc * nb, who = q / nb, j = q - who * nb;
      const long e = e0 + el;
      const long src = who == 0 ? e : nbr[(size_t)e * nf + who - 1];
      xs[t] = x[(size_t)src * nb + j];
    }
    __syncthreads();
    if (sub < nl) {
      const long e = e0 + sub;
      const unsigned short* base = (b == 0 ? Dm + (size_t)e * bstride : O + ((size_t)e * nf + b - 1) * bstride) +
                                   8 * tt;
      const float* xb = xs + ((size_t)sub * nsrc + b) * nb;
      float acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll 8
      for (int c = 0; c < nb; ++c) {
        float a[8];
        ld_bf16x8(base + (size_t)c * ld16, a);
        const float xv = xb[c];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += a[j] * xv;
      }
      float* pr = part + ((size_t)sub * nsrc + b) * ld16 + 8 * tt;
#pragma unroll
      for (int j = 0; j < 8; ++j) pr[j] = acc[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
      const int el = t / nb, row = t - el * nb;
      const float* pe = part + (size_t)el * nsrc * ld16 + row;
      float sum = 0.f;
      for (int bb = 0; bb < nsrc; ++bb) sum += pe[(size_t)bb * ld16];
      y[(size_t)(e0 + el) * nb + row] = sum;
    }
    __syncthreads();
  }
}

cudaError_t launch_bsr_bf16(const unsigned short* D, const unsigned short* O, const int* nbr, int nf,
                            const float* x, float* y, int nb, int E, cudaStream_t st) {
  const int ld16 = ld_bf16(nb), tpe = ld16 / 8, tpb = (1 + nf) * tpe;
  if (tpb > 256) return cudaErrorInvalidValue;   // the level cannot use BF16 blocks (checked at setup)
  const int epc = std::max(1, 256 / tpb);
  const int threads = (epc * tpb + 31) / 32 * 32;
  const int grid = std::min((E + epc - 1) / epc, 16 * num_sms());
  const size_t smem = (size_t)epc * (1 + nf) * (nb + ld16) * sizeof(float);
  note_launch();
  bsr_bf16_kernel<<<grid, threads, smem, st>>>(D, O, nbr, nf, x, y, nb, ld16, E, epc, tpe);
  return cudaGetLastError();
}

}  // namespace dgk
