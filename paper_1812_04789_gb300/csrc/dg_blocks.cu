// Element Jacobian blocks, subspace inheritance and block Jacobi
// (Sec. 5.1 eq. ODEDG; Sec. 6.1 inheritance; Sec. 6.3 element block Jacobi).
//
// probe_kernel: one CTA per element (grid-stride).  The element's and its 2d
// neighbours' traces are computed once; then for every local unit direction
// e_j (variable w, mode i) the pointwise physics is evaluated in dual numbers
// with the tangent phi_i (grad phi_i) in component w, and projected onto all
// test functions: column j of dR_e/dW_e.  Faces are evaluated from the
// element's own side (each interior face twice over the mesh), so no face
// slots are needed.  Neighbour blocks dR_e/dW_nbr take the seed on the
// neighbour's trace instead, for the first nmc modes only (Sec. 6.3: at
// coarse order).  A direction with a single element makes the element its own
// neighbour: the seed then sits on both traces and the coupling belongs to
// the diagonal block (the neighbour block is zero).
#include <algorithm>
#include <type_traits>

#include "dg_internal.h"

namespace dgk {

template <class T>
struct ProbeLayout {
  size_t cW, cU, cFU, bF, bG, bFp, bDo, total;
  __host__ __device__ ProbeLayout(int D, int nb, int nq, int nqf) {
    int M = D + 2, nf = 2 * D;
    size_t o = 0;
    cW = o;  o += (size_t)(1 + nf) * nb;
    cU = o;  o += (size_t)nq * M * (1 + D);
    cFU = o; o += (size_t)nf * 2 * nqf * M * (1 + D);
    bF = o;  o += (size_t)nq * M * D;
    bG = o;  o += (size_t)nf * 2 * nqf * M;
    bFp = o; o += (size_t)nf * nqf * M;
    bDo = o; o += (size_t)nf * nqf * M * D;
    total = o;
  }
};

template <int D, class T>
__device__ __forceinline__ void face_point_tangent(const T* pu_own, const T* pu_nb, int k, int side,
                                                   int w, T so, const T* sgo, T sn, const T* sgn,
                                                   const Phys<T>& ph, T* bGL, T* bGR, T* bFp,
                                                   T* bDo) {
  using S = Dual<T>;
  constexpr int M = D + 2;
  // pu_*: primal [M] then grad [M][D]; seeds so/sgo on own trace, sn/sgn on the neighbour's
  S uo[M], un[M], go[M][D], gn[M][D];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    uo[v] = S(pu_own[v], v == w ? so : T(0));
    un[v] = S(pu_nb[v], v == w ? sn : T(0));
#pragma unroll
    for (int kk = 0; kk < D; ++kk) {
      go[v][kk] = S(pu_own[M + v * D + kk], v == w ? sgo[kk] : T(0));
      gn[v][kk] = S(pu_nb[M + v * D + kk], v == w ? sgn[kk] : T(0));
    }
  }
  S fp[M], GLn[M], GRn[M], DL[M][D], DR[M][D];
  if (side)
    face_point_k<D, S, T>(k, uo, go, un, gn, ph, fp, GLn, GRn, DL, DR);
  else
    face_point_k<D, S, T>(k, un, gn, uo, go, ph, fp, GLn, GRn, DL, DR);
#pragma unroll
  for (int v = 0; v < M; ++v) {
    bFp[v] = tan_part(fp[v]);
    bGL[v] = tan_part(GLn[v]);
    bGR[v] = tan_part(GRn[v]);
#pragma unroll
    for (int kk = 0; kk < D; ++kk) bDo[v * D + kk] = tan_part(side ? DL[v][kk] : DR[v][kk]);
  }
}

template <int D, class T>
__global__ void __launch_bounds__(256) probe_kernel(MeshView<T> mv, Phys<T> ph, const T* __restrict__ W,
                                                    T sigma, T* __restrict__ Dout, T* __restrict__ Oout,
                                                    int nmc, T* gscratch, int use_smem, int* status) {
  constexpr int M = D + 2, NF = 2 * D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, nqf = mv.nqf, E = mv.E;
  ProbeLayout<T> L(D, nb, nq, nqf);
  T* C = use_smem ? reinterpret_cast<T*>(smem_raw) : gscratch + (size_t)blockIdx.x * L.total;
  T* cW = C + L.cW;
  T* cU = C + L.cU;
  T* cFU = C + L.cFU;
  T* bF = C + L.bF;
  T* bG = C + L.bG;
  T* bFp = C + L.bFp;
  T* bDo = C + L.bDo;
  const int PU = M * (1 + D);
  const int nbc = M * nmc;
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    int nbrs[NF];
#pragma unroll
    for (int s = 0; s < NF; ++s) nbrs[s] = mv.nbr[e * NF + s];
    // ---- stage W of the element and its neighbours (face order s = 2k + side)
    for (int t = threadIdx.x; t < (1 + NF) * nb; t += blockDim.x) {
      int who = t / nb, j = t % nb;
      int el = who == 0 ? e : nbrs[who - 1];
      cW[t] = W[(size_t)el * nb + j];
    }
    __syncthreads();
    // ---- primal traces: volume points and both sides of every face
    for (int t = threadIdx.x; t < nq + NF * 2 * nqf; t += blockDim.x) {
      T u[M], g[M][D];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        u[v] = T(0);
#pragma unroll
        for (int kk = 0; kk < D; ++kk) g[v][kk] = T(0);
      }
      T* dst;
      if (t < nq) {
        int q = t;
        for (int i = 0; i < nm; ++i) {
          T p = mv.vphiT[(size_t)i * nq + q];
#pragma unroll
          for (int v = 0; v < M; ++v) {
            T a = cW[v * nm + i];
            u[v] += a * p;
#pragma unroll
            for (int kk = 0; kk < D; ++kk) g[v][kk] += a * mv.vdphiT[((size_t)kk * nm + i) * nq + q];
          }
        }
        dst = cU + (size_t)q * PU;
      } else {
        int r = t - nq, s = r / (2 * nqf), who = (r / nqf) % 2, q = r % nqf;
        int lf = who == 0 ? s : (s ^ 1);               // own face s, neighbour's face s^1
        const T* ws = cW + (size_t)(who == 0 ? 0 : 1 + s) * nb;
        for (int i = 0; i < nm; ++i) {
          T p = mv.fphiT[((size_t)lf * nm + i) * nqf + q];
#pragma unroll
          for (int v = 0; v < M; ++v) {
            T a = ws[v * nm + i];
            u[v] += a * p;
#pragma unroll
            for (int kk = 0; kk < D; ++kk)
              g[v][kk] += a * mv.fdphiT[(((size_t)lf * D + kk) * nm + i) * nqf + q];
          }
        }
        dst = cFU + (size_t)r * PU;
      }
      if (!physical<D>(u, (double)ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
#pragma unroll
      for (int v = 0; v < M; ++v) {
        dst[v] = u[v];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) dst[M + v * D + kk] = g[v][kk];
      }
    }
    __syncthreads();
    // ---- diagonal block, one column per local unit direction
    for (int jj = 0; jj < nb; ++jj) {
      const int w = jj / nm, i = jj % nm;
      for (int t = threadIdx.x; t < nq + NF * nqf; t += blockDim.x) {
        if (t < nq) {
          int q = t;
          using S = Dual<T>;
          const T* pu = cU + (size_t)q * PU;
          S u[M], g[M][D];
          T p = mv.vphi[(size_t)q * nm + i];
#pragma unroll
          for (int v = 0; v < M; ++v) {
            u[v] = S(pu[v], v == w ? p : T(0));
#pragma unroll
            for (int kk = 0; kk < D; ++kk)
              g[v][kk] = S(pu[M + v * D + kk], v == w ? mv.vdphi[((size_t)kk * nq + q) * nm + i] : T(0));
          }
          S F[M][D];
          flux_total<D, S, T>(u, g, F, ph);
          T wq = mv.vw[q];
#pragma unroll
          for (int v = 0; v < M; ++v)
#pragma unroll
            for (int kk = 0; kk < D; ++kk) bF[((size_t)q * M + v) * D + kk] = wq * F[v][kk].d;
        } else {
          int r = t - nq, s = r / nqf, q = r % nqf;
          int k = s / 2, side = s % 2;
          bool self = nbrs[s] == e;
          T so = mv.fphi[((size_t)s * nqf + q) * nm + i];
          T sgo[D], sgn[D];
          T sn = self ? mv.fphi[((size_t)(s ^ 1) * nqf + q) * nm + i] : T(0);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) {
            sgo[kk] = mv.fdphi[(((size_t)s * D + kk) * nqf + q) * nm + i];
            sgn[kk] = self ? mv.fdphi[(((size_t)(s ^ 1) * D + kk) * nqf + q) * nm + i] : T(0);
          }
          face_point_tangent<D, T>(cFU + ((size_t)(s * 2) * nqf + q) * PU,
                                   cFU + ((size_t)(s * 2 + 1) * nqf + q) * PU, k, side, w, so, sgo,
                                   sn, sgn, ph, bG + ((size_t)(s * 2) * nqf + q) * M,
                                   bG + ((size_t)(s * 2 + 1) * nqf + q) * M,
                                   bFp + ((size_t)s * nqf + q) * M, bDo + ((size_t)s * nqf + q) * M * D);
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < NF * nqf; t += blockDim.x) {
        int s = t / nqf, q = t % nqf, k = s / 2;
        const T* PL = mv.lift + ((size_t)(2 * k + 1) * nqf + q) * nqf;
        const T* PR = mv.lift + ((size_t)(2 * k) * nqf + q) * nqf;
        T dl[M], dr[M];
#pragma unroll
        for (int v = 0; v < M; ++v) dl[v] = dr[v] = T(0);
        for (int q2 = 0; q2 < nqf; ++q2) {
          const T* gl = bG + ((size_t)(s * 2) * nqf + q2) * M;
          const T* gr = bG + ((size_t)(s * 2 + 1) * nqf + q2) * M;
#pragma unroll
          for (int v = 0; v < M; ++v) {
            dl[v] += PL[q2] * gl[v];
            dr[v] += PR[q2] * gr[v];
          }
        }
        T* fo = bFp + ((size_t)s * nqf + q) * M;
#pragma unroll
        for (int v = 0; v < M; ++v) fo[v] += ph.eta * T(0.5) * (dl[v] + dr[v]);
      }
      __syncthreads();
      for (int r = threadIdx.x; r < nb; r += blockDim.x) {
        int v = r / nm, ip = r % nm;
        T acc = T(0);
        for (int q = 0; q < nq; ++q) {
          const T* fq = bF + ((size_t)q * M + v) * D;
#pragma unroll
          for (int kk = 0; kk < D; ++kk) acc -= mv.vdphi[((size_t)kk * nq + q) * nm + ip] * fq[kk];
        }
#pragma unroll
        for (int s = 0; s < NF; ++s) {
          int k = s / 2;
          T sg = (s % 2) ? T(1) : T(-1);
          const T* fw = mv.fw + (size_t)k * nqf;
          T a2 = T(0);
          for (int q = 0; q < nqf; ++q) {
            T x = sg * mv.fphi[((size_t)s * nqf + q) * nm + ip] * bFp[((size_t)s * nqf + q) * M + v];
#pragma unroll
            for (int kk = 0; kk < D; ++kk)
              x -= mv.fdphi[(((size_t)s * D + kk) * nqf + q) * nm + ip] * bDo[(((size_t)s * nqf + q) * M + v) * D + kk];
            a2 += fw[q] * x;
          }
          acc += a2;
        }
        if (r == jj) acc += sigma * mv.detJ;
        Dout[((size_t)e * nb + r) * nb + jj] = acc;
      }
      __syncthreads();
    }
    // ---- neighbour blocks at coarse order (seed on the neighbour's trace)
    if (Oout != nullptr) {
      for (int jc = 0; jc < nbc; ++jc) {
        const int w = jc / nmc, i = jc % nmc;
        for (int t = threadIdx.x; t < NF * nqf; t += blockDim.x) {
          int s = t / nqf, q = t % nqf, k = s / 2, side = s % 2;
          T sgo[D], sgn[D];
          T sn = mv.fphi[((size_t)(s ^ 1) * nqf + q) * nm + i];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) {
            sgo[kk] = T(0);
            sgn[kk] = mv.fdphi[(((size_t)(s ^ 1) * D + kk) * nqf + q) * nm + i];
          }
          face_point_tangent<D, T>(cFU + ((size_t)(s * 2) * nqf + q) * PU,
                                   cFU + ((size_t)(s * 2 + 1) * nqf + q) * PU, k, side, w, T(0), sgo,
                                   sn, sgn, ph, bG + ((size_t)(s * 2) * nqf + q) * M,
                                   bG + ((size_t)(s * 2 + 1) * nqf + q) * M,
                                   bFp + ((size_t)s * nqf + q) * M, bDo + ((size_t)s * nqf + q) * M * D);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NF * nqf; t += blockDim.x) {
          int s = t / nqf, q = t % nqf, k = s / 2;
          const T* PL = mv.lift + ((size_t)(2 * k + 1) * nqf + q) * nqf;
          const T* PR = mv.lift + ((size_t)(2 * k) * nqf + q) * nqf;
          T dl[M], dr[M];
#pragma unroll
          for (int v = 0; v < M; ++v) dl[v] = dr[v] = T(0);
          for (int q2 = 0; q2 < nqf; ++q2) {
            const T* gl = bG + ((size_t)(s * 2) * nqf + q2) * M;
            const T* gr = bG + ((size_t)(s * 2 + 1) * nqf + q2) * M;
#pragma unroll
            for (int v = 0; v < M; ++v) {
              dl[v] += PL[q2] * gl[v];
              dr[v] += PR[q2] * gr[v];
            }
          }
          T* fo = bFp + ((size_t)s * nqf + q) * M;
#pragma unroll
          for (int v = 0; v < M; ++v) fo[v] += ph.eta * T(0.5) * (dl[v] + dr[v]);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NF * nbc; t += blockDim.x) {
          int s = t / nbc, rc = t % nbc, v = rc / nmc, ip = rc % nmc, k = s / 2;
          T sg = (s % 2) ? T(1) : T(-1);
          const T* fw = mv.fw + (size_t)k * nqf;
          T acc = T(0);
          for (int q = 0; q < nqf; ++q) {
            T x = sg * mv.fphi[((size_t)s * nqf + q) * nm + ip] * bFp[((size_t)s * nqf + q) * M + v];
#pragma unroll
            for (int kk = 0; kk < D; ++kk)
              x -= mv.fdphi[(((size_t)s * D + kk) * nqf + q) * nm + ip] * bDo[(((size_t)s * nqf + q) * M + v) * D + kk];
            acc += fw[q] * x;
          }
          if (nbrs[s] == e) acc = T(0);
          Oout[(((size_t)e * NF + s) * nbc + rc) * nbc + jc] = acc;
        }
        __syncthreads();
      }
    }
  }
}

template <class T>
size_t probe_scratch_elems(const Mesh& M, int nmc, bool* fits_smem) {
  (void)nmc;
  ProbeLayout<T> L(M.d, M.nb, M.nq, M.nqf);
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
static cudaError_t run_probe(const Mesh& Ms, const T* W, T sigma, T* Dout, T* Oout, int nmc, T* scratch,
                             size_t scratch_elems, cudaStream_t st) {
  bool fits;
  size_t tot = probe_scratch_elems<T>(Ms, nmc, &fits);
  int grid;
  size_t smem = 0;
  if (fits) {
    smem = tot * sizeof(T);
    grid = Ms.E;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(probe_kernel<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  } else {
    grid = std::min(Ms.E, probe_grid_global());
    if (!scratch || scratch_elems < tot * (size_t)grid) return cudaErrorInvalidValue;
  }
  note_launch();
  probe_kernel<D, T><<<grid, 256, smem, st>>>(Ms.view<T>(), Ms.phys_t<T>(), W, sigma, Dout, Oout, nmc,
                                             scratch, fits ? 1 : 0, Ms.status);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_probe_blocks(const Mesh& M, const T* W, T sigma, T* D, T* O, int nmc, T* scratch,
                                size_t scratch_elems, cudaStream_t st) {
  if (M.d == 2) return run_probe<2, T>(M, W, sigma, D, O, nmc, scratch, scratch_elems, st);
  return run_probe<3, T>(M, W, sigma, D, O, nmc, scratch, scratch_elems, st);
}
template cudaError_t launch_probe_blocks<double>(const Mesh&, const double*, double, double*, double*, int,
                                                 double*, size_t, cudaStream_t);
template cudaError_t launch_probe_blocks<float>(const Mesh&, const float*, float, float*, float*, int, float*,
                                                size_t, cudaStream_t);

// ---------------------------------------------------------------- block inverse
// In-place Gauss-Jordan inversion with partial (row) pivoting: the largest
// |entry| of the pivot column, the lowest row index on ties; the row swaps
// are undone on the columns of the inverse at the end.  A zero pivot marks the
// status word and leaves the block unusable.
template <class T>
__global__ void __launch_bounds__(256) block_inverse_kernel(T* __restrict__ blocks, int nb, long nblk,
                                                            int use_smem, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // byte layout: rv[blockDim] doubles | colk[nb] | prow[nb] | ri[blockDim] | perm[nb] | A (16-aligned)
  double* rv = reinterpret_cast<double*>(smem_raw);
  T* colk = reinterpret_cast<T*>(rv + blockDim.x);
  T* prow = colk + nb;
  int* ri = reinterpret_cast<int*>(prow + nb);
  int* perm = ri + blockDim.x;
  T* As = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(perm + nb) + 15) & ~uintptr_t(15));
  const int nn = nb * nb;
  for (long b = blockIdx.x; b < nblk; b += gridDim.x) {
    T* Ag = blocks + (size_t)b * nn;
    T* A = use_smem ? As : Ag;
    if (use_smem) {
      for (int t = threadIdx.x; t < nn; t += blockDim.x) A[t] = Ag[t];
      __syncthreads();
    }
    bool bad = false;
    for (int k = 0; k < nb; ++k) {
      // pivot search
      double best = -1.0;
      int bi = nb;
      for (int i = k + threadIdx.x; i < nb; i += blockDim.x) {
        double a = fabs((double)A[(size_t)i * nb + k]);
        if (a > best || (a == best && i < bi)) {
          best = a;
          bi = i;
        }
      }
      rv[threadIdx.x] = best;
      ri[threadIdx.x] = bi;
      __syncthreads();
      for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
          double a = rv[threadIdx.x + s];
          int ia = ri[threadIdx.x + s];
          if (a > rv[threadIdx.x] || (a == rv[threadIdx.x] && ia < ri[threadIdx.x])) {
            rv[threadIdx.x] = a;
            ri[threadIdx.x] = ia;
          }
        }
        __syncthreads();
      }
      int p = ri[0];
      double pa = rv[0];
      __syncthreads();
      if (!(pa > 0.0) || p >= nb) {
        bad = true;
        p = k;
      }
      if (threadIdx.x == 0) perm[k] = p;
      if (p != k)
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
          T x = A[(size_t)k * nb + j];
          A[(size_t)k * nb + j] = A[(size_t)p * nb + j];
          A[(size_t)p * nb + j] = x;
        }
      __syncthreads();
      T piv = A[(size_t)k * nb + k];
      if (bad) piv = T(1);
      T ipiv = T(1) / piv;
      for (int j = threadIdx.x; j < nb; j += blockDim.x) prow[j] = (j == k ? T(1) : A[(size_t)k * nb + j]) * ipiv;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) colk[i] = (i == k) ? T(0) : A[(size_t)i * nb + k];
      __syncthreads();
      for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        int i = t / nb, j = t % nb;
        if (i == k) {
          A[t] = prow[j];
        } else {
          T a = (j == k) ? T(0) : A[t];
          A[t] = a - colk[i] * prow[j];
        }
      }
      __syncthreads();
    }
    // undo the row interchanges on the columns, last first
    for (int k = nb - 1; k >= 0; --k) {
      int p = perm[k];
      if (p != k)
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
          T x = A[(size_t)i * nb + k];
          A[(size_t)i * nb + k] = A[(size_t)i * nb + p];
          A[(size_t)i * nb + p] = x;
        }
      __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicOr(status, ST_SINGULAR);
    if (use_smem) {
      for (int t = threadIdx.x; t < nn; t += blockDim.x) Ag[t] = A[t];
    }
    __syncthreads();
  }
}

template <class T>
cudaError_t launch_block_inverse(T* A, int nb, long nblk, int* status, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  const int threads = 256;
  size_t base = (2 * nb + 2) * sizeof(T) + threads * (sizeof(double) + sizeof(int)) + (nb + 4) * sizeof(int) + 32;
  size_t full = base + (size_t)nb * nb * sizeof(T);
  int use_smem = full <= 200 * 1024;
  size_t smem = use_smem ? full : base;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(block_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  long grid = std::min<long>(nblk, 16L * num_sms());
  note_launch();
  block_inverse_kernel<T><<<(int)grid, threads, smem, st>>>(A, nb, nblk, use_smem, status);
  return cudaGetLastError();
}
template cudaError_t launch_block_inverse<double>(double*, int, long, int*, cudaStream_t);
template cudaError_t launch_block_inverse<float>(float*, int, long, int*, cudaStream_t);

// ---------------------------------------------------------------- truncation
template <class T>
__global__ void truncate_kernel(const T* __restrict__ src, int nms, T* __restrict__ dst, int nmt, int m,
                                long nblk) {
  const int nbs = m * nms, nbt = m * nmt;
  const long tot = nblk * nbt * nbt;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    long b = t / ((long)nbt * nbt);
    int r = (int)(t % ((long)nbt * nbt));
    int row = r / nbt, col = r % nbt;
    int v = row / nmt, i = row % nmt, w = col / nmt, j = col % nmt;
    dst[t] = src[(size_t)b * nbs * nbs + (size_t)(v * nms + i) * nbs + (w * nms + j)];
  }
}

template <class T>
cudaError_t launch_truncate_blocks(const T* src, int nms, T* dst, int nmt, int m, long nblk, cudaStream_t st) {
  long tot = nblk * (long)(m * nmt) * (m * nmt);
  if (tot <= 0) return cudaSuccess;
  long grid = std::min<long>((tot + 255) / 256, 65535L * 8);
  note_launch();
  truncate_kernel<T><<<(int)grid, 256, 0, st>>>(src, nms, dst, nmt, m, nblk);
  return cudaGetLastError();
}
template cudaError_t launch_truncate_blocks<double>(const double*, int, double*, int, int, long, cudaStream_t);
template cudaError_t launch_truncate_blocks<float>(const float*, int, float*, int, int, long, cudaStream_t);

// ---------------------------------------------------------------- block apply / BSR
// One CTA per element: the element's input (and neighbours' for BSR) staged in
// shared memory, one warp per block row with the lanes striding the columns
// (coalesced row reads), fixed butterfly reduction.
template <class T>
__global__ void __launch_bounds__(256) bsr_kernel(const T* __restrict__ Dm, const T* __restrict__ O,
                                                  const int* __restrict__ nbr, int nf, const T* __restrict__ x,
                                                  T* __restrict__ y, int nb, int E) {
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
    for (int r = warp; r < nb; r += nw) {
      T acc = T(0);
      const T* Ar = Dm + ((size_t)e * nb + r) * nb;
      for (int c = lane; c < nb; c += 32) acc += Ar[c] * xs[c];
      if (O) {
        for (int s = 0; s < nf; ++s) {
          const T* Orow = O + (((size_t)e * nf + s) * nb + r) * nb;
          const T* xn = xs + (size_t)(1 + s) * nb;
          for (int c = lane; c < nb; c += 32) acc += Orow[c] * xn[c];
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) y[(size_t)e * nb + r] = acc;
    }
    __syncthreads();
  }
}

template <class T>
cudaError_t launch_block_apply(const T* A, const T* r, T* z, int nb, int E, cudaStream_t st) {
  int grid = std::min(E, 32 * num_sms());
  note_launch();
  bsr_kernel<T><<<grid, 256, nb * sizeof(T), st>>>(A, nullptr, nullptr, 0, r, z, nb, E);
  return cudaGetLastError();
}
template cudaError_t launch_block_apply<double>(const double*, const double*, double*, int, int, cudaStream_t);
template cudaError_t launch_block_apply<float>(const float*, const float*, float*, int, int, cudaStream_t);

template <class T>
cudaError_t launch_bsr(const T* D, const T* O, const int* nbr, int d, const T* x, T* y, int nb, int E,
                       cudaStream_t st) {
  int grid = std::min(E, 32 * num_sms());
  size_t smem = (size_t)(1 + 2 * d) * nb * sizeof(T);
  note_launch();
  bsr_kernel<T><<<grid, 256, smem, st>>>(D, O, nbr, 2 * d, x, y, nb, E);
  return cudaGetLastError();
}
template cudaError_t launch_bsr<double>(const double*, const double*, const int*, int, const double*, double*,
                                        int, int, cudaStream_t);
template cudaError_t launch_bsr<float>(const float*, const float*, const int*, int, const float*, float*, int,
                                       int, cudaStream_t);

}  // namespace dgk
