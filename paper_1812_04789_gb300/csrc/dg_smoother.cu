// Persistent GMRES(BJ) smoother of the inherited coarse levels: one
// cooperative launch runs a whole SMOOTH / SOLVE call of Algorithm 2 (nu
// iterations of GMRES right-preconditioned by element block Jacobi, Sec. 6.3,
// on the inherited block-sparse operator of Sec. 6.1), where the
// launch-per-operation path takes about eleven small kernels per iteration.
//
// Work split: CTA c owns a contiguous range of elements for the whole call
// (its rows of every vector).  Per iteration j:
//   A  v_j = w / ||w|| (own rows); z_j = D^{-1} v_j (own elements)      | grid barrier
//   B  w = A z_j (own elements, neighbours' z_j read); partial V^T w    | grid barrier
//   C  h1 = sum of partials; w -= V h1; partial V^T w                    | grid barrier
//   D  h2 = sum of partials; w -= V h2; partial ||w||^2                  | grid barrier
// (CGS2, as the launch-per-operation Arnoldi).  Every CTA sums the partials
// of all CTAs in the same fixed order and keeps its own copy of the
// Hessenberg matrix, the Givens rotations and g, so all CTAs hold identical
// scalars and the final x += Z y needs no further barrier.
//
// The grid barrier is a counter in device memory, zeroed before the launch:
// barrier k waits until k * expect CTAs have arrived.  Every wait is bounded
// (2 s of the global timer): on expiry the CTA sets ST_TIMEOUT in the mesh
// status word and returns, and the other CTAs see the flag while they wait
// and return too; a launch that finds ST_TIMEOUT already set returns at once.
// A handle whose status shows ST_TIMEOUT has an unfinished smoother result:
// the application is untrusted until the status is cleared (dg_status_sync)
// and the preconditioner refreshed.
#include <math.h>

#include <algorithm>

#include "dg_internal.h"

namespace dgk {

// R consecutive rows of one column of a column-major block from 16 bytes.
template <class S>
struct Col16;
template <>
struct Col16<float> {
  static constexpr int R = 4;
  __device__ __forceinline__ static void load(const float* p, float* v) {
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "l"(p));
  }
};
template <>
struct Col16<unsigned short> {
  static constexpr int R = 8;
  __device__ __forceinline__ static void load(const unsigned short* p, float* v) { ld_bf16x8(p, v); }
};

template <class S>
struct CoopArgs {
  const S* Dinv;        // inverse diagonal blocks, column-major, leading dimension ld, nb * ld apart
  const S* Dop;         // inherited diagonal blocks (same layout)
  const S* O;           // inherited neighbour blocks [E][nf] (same layout)
  const int* nbr;       // [E][nf]
  const float* b;
  float* x;
  float* V;             // (nu + 1) x N
  float* Z;             // nu x N
  float* w;             // N
  double* part;         // [grid][2 (nu + 1) + 1]
  unsigned* bar;        // barrier counter, zero at launch
  int* status;          // mesh status word (ST_TIMEOUT)
  int* kflag;           // Krylov status bits (ST_NONFINITE)
  long N;
  int nu, nb, ld, nf, E, chunk, epc, tpe, expect;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier number k (target k * expect arrivals); false when a wait
// ran out here or elsewhere (ST_TIMEOUT), and then the caller returns.
__device__ bool grid_barrier(unsigned* bar, unsigned target, int* status, int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned long long t0 = global_ns();
    int ok = 1;
    while (*(volatile unsigned*)bar < target) {
      if (*(volatile int*)status & ST_TIMEOUT) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > 2000000000ull) {
        atomicOr(status, ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// sum over the CTA's threads of s, returned to every thread (red: 32 doubles)
__device__ double block_sum(double s, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = s;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// out[i] = sum over the CTA's rows [n0, n1) of V_i . w, i < nv (warp per i)
__device__ void own_dots(int nv, const float* V, long N, const float* w, long n0, long n1, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < nv; i += nw) {
    const float* v = V + (size_t)i * N;
    double s = 0.0;
    for (long n = n0 + lane; n < n1; n += 32) s += (double)v[n] * (double)w[n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
  }
}

// dst[i] = sum over CTAs c = 0..G-1 of part[c * stride + i], i < nv, in a
// fixed order (the same in every CTA); partials of other CTAs read past L1
__device__ void sum_parts(int nv, const double* part, int stride, int G, double* dst) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < nv; i += nw) {
    double s = 0.0;
    for (int c = lane; c < G; c += 32) s += __ldcg(part + (size_t)c * stride + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dst[i] = s;
  }
  __syncthreads();
}

// out_e = [bsub_e -] (D_e in_e + sum_s O_{e,s} in_nbr(e,s)) for e in [e_beg, e_end):
// a thread per (element, block, R rows), partial rows summed in a fixed order.
template <class S>
__device__ void bsr_own(const CoopArgs<S>& a, const float* in, float* out, const float* bsub, int e_beg, int e_end,
                        float* xs, float* pt) {
  constexpr int R = Col16<S>::R;
  const int nb = a.nb, ld = a.ld, nf = a.nf, nsrc = 1 + nf, tpb = nsrc * a.tpe;
  const size_t bs = (size_t)nb * ld;
  const int sub = threadIdx.x / tpb, r = threadIdx.x - sub * tpb, blk = r / a.tpe, tt = r - blk * a.tpe;
  for (int e0 = e_beg; e0 < e_end; e0 += a.epc) {
    const int nl = min(a.epc, e_end - e0);
    for (int t = threadIdx.x; t < nl * nsrc * nb; t += blockDim.x) {
      const int el = t / (nsrc * nb), q = t - el * nsrc * nb, who = q / nb, j = q - who * nb;
      const int e = e0 + el;
      const int src = who == 0 ? e : a.nbr[(size_t)e * nf + who - 1];
      xs[t] = __ldcg(in + (size_t)src * nb + j);
    }
    __syncthreads();
    if (sub < nl) {
      const int e = e0 + sub;
      const S* base = (blk == 0 ? a.Dop + (size_t)e * bs : a.O + ((size_t)e * nf + blk - 1) * bs) + R * tt;
      const float* xb = xs + ((size_t)sub * nsrc + blk) * nb;
      float acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = 0.f;
#pragma unroll 8
      for (int c = 0; c < nb; ++c) {
        float v[R];
        Col16<S>::load(base + (size_t)c * ld, v);
        const float xv = xb[c];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += v[j] * xv;
      }
      float* p = pt + ((size_t)sub * nsrc + blk) * ld + R * tt;
#pragma unroll
      for (int j = 0; j < R; ++j) p[j] = acc[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
      const int el = t / nb, row = t - el * nb;
      const float* pe = pt + (size_t)el * nsrc * ld + row;
      float s = 0.f;
      for (int bb = 0; bb < nsrc; ++bb) s += pe[(size_t)bb * ld];
      const size_t n = (size_t)(e0 + el) * nb + row;
      out[n] = bsub ? bsub[n] - s : s;
    }
    __syncthreads();
  }
}

// z_e = D_e^{-1} v_e for e in [e_beg, e_end) (own rows only)
template <class S>
__device__ void bj_own(const CoopArgs<S>& a, const float* v, float* z, int e_beg, int e_end, float* xs) {
  constexpr int R = Col16<S>::R;
  const int nb = a.nb, ld = a.ld, tpe = a.tpe, epc = blockDim.x / tpe;
  const size_t bs = (size_t)nb * ld;
  const int sub = threadIdx.x / tpe, tt = threadIdx.x - sub * tpe;
  for (int e0 = e_beg; e0 < e_end; e0 += epc) {
    const int nl = min(epc, e_end - e0);
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) xs[t] = v[(size_t)e0 * nb + t];
    __syncthreads();
    if (sub < nl) {
      const S* base = a.Dinv + (size_t)(e0 + sub) * bs + R * tt;
      const float* xe = xs + (size_t)sub * nb;
      float acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = 0.f;
#pragma unroll 8
      for (int c = 0; c < nb; ++c) {
        float m[R];
        Col16<S>::load(base + (size_t)c * ld, m);
        const float xv = xe[c];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += m[j] * xv;
      }
      float* zo = z + (size_t)(e0 + sub) * nb + R * tt;
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (R * tt + j < nb) zo[j] = acc[j];
    }
    __syncthreads();
  }
}

template <class S>
__global__ void __launch_bounds__(256) coop_smooth_kernel(CoopArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nu = a.nu, ldh = nu + 1;
  double* H = reinterpret_cast<double*>(smem_raw);   // (nu + 1) x nu, column-major
  double* cs = H + (size_t)ldh * nu;
  double* sn = cs + nu;
  double* g = sn + nu;                                // nu + 1
  double* h1 = g + ldh;                               // nu + 1
  double* h2 = h1 + ldh;                              // nu + 1
  double* red = h2 + ldh;                             // 32
  int* sflag = reinterpret_cast<int*>(red + 32);      // 4 ints
  float* xs = reinterpret_cast<float*>(sflag + 4);
  const int nsrc = 1 + a.nf;
  float* pt = xs + std::max((size_t)a.epc * nsrc * a.nb, (size_t)(blockDim.x / a.tpe) * a.nb);

  const int G = gridDim.x, stride = 2 * ldh + 1;
  double* mypart = a.part + (size_t)blockIdx.x * stride;   // [0, ldh): pass 1, [ldh, 2 ldh): pass 2, last: norm
  const int e_beg = min(a.E, (int)blockIdx.x * a.chunk), e_end = min(a.E, e_beg + a.chunk);
  const long n0 = (long)e_beg * a.nb, n1 = (long)e_end * a.nb;
  const long N = a.N;
  unsigned nbar = 0;

  if (threadIdx.x == 0) sflag[1] = (*(volatile int*)a.status & ST_TIMEOUT) ? 1 : 0;
  __syncthreads();
  if (sflag[1]) return;   // an earlier wait ran out: leave x as it is

  // r = b - A x into w, ||r||^2
  bsr_own<S>(a, a.x, a.w, a.b, e_beg, e_end, xs, pt);
  {
    double s = 0.0;
    for (long n = n0 + threadIdx.x; n < n1; n += blockDim.x) s += (double)a.w[n] * (double)a.w[n];
    s = block_sum(s, red);
    if (threadIdx.x == 0) mypart[2 * ldh] = s;
  }
  if (!grid_barrier(a.bar, ++nbar * a.expect, a.status, sflag)) return;
  sum_parts(1, a.part + 2 * ldh, stride, G, h2);
  const double beta = sqrt(h2[0]);
  if (!(beta > 0.0) || !isfinite(beta)) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !isfinite(beta)) atomicOr(a.kflag, ST_NONFINITE);
    return;   // b - A x = 0 (or not finite): nothing to smooth
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < ldh; ++i) g[i] = 0.0;
    g[0] = beta;
  }
  double inv = 1.0 / beta;
  int kdone = 0;
  for (int j = 0; j < nu; ++j) {
    // A: v_j = w / ||w||, z_j = D^{-1} v_j
    float* vj = a.V + (size_t)j * N;
    float* zj = a.Z + (size_t)j * N;
    for (long n = n0 + threadIdx.x; n < n1; n += blockDim.x) vj[n] = (float)(inv * (double)a.w[n]);
    __syncthreads();
    bj_own<S>(a, vj, zj, e_beg, e_end, xs);
    if (!grid_barrier(a.bar, ++nbar * a.expect, a.status, sflag)) return;
    // B: w = A z_j, first pass of inner products
    bsr_own<S>(a, zj, a.w, nullptr, e_beg, e_end, xs, pt);
    own_dots(j + 1, a.V, N, a.w, n0, n1, mypart);
    if (!grid_barrier(a.bar, ++nbar * a.expect, a.status, sflag)) return;
    // C: w -= V h1, second pass
    sum_parts(j + 1, a.part, stride, G, h1);
    for (long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
      double acc = (double)a.w[n];
      for (int i = 0; i <= j; ++i) acc -= h1[i] * (double)a.V[(size_t)i * N + n];
      a.w[n] = (float)acc;
    }
    __syncthreads();
    own_dots(j + 1, a.V, N, a.w, n0, n1, mypart + ldh);
    if (!grid_barrier(a.bar, ++nbar * a.expect, a.status, sflag)) return;
    // D: w -= V h2, ||w||^2
    sum_parts(j + 1, a.part + ldh, stride, G, h2);
    double s = 0.0;
    for (long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
      double acc = (double)a.w[n];
      for (int i = 0; i <= j; ++i) acc -= h2[i] * (double)a.V[(size_t)i * N + n];
      const float wf = (float)acc;
      a.w[n] = wf;
      s += (double)wf * (double)wf;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) mypart[2 * ldh] = s;
    if (!grid_barrier(a.bar, ++nbar * a.expect, a.status, sflag)) return;
    sum_parts(1, a.part + 2 * ldh, stride, G, red + 16);   // red[16] = ||w||^2 (red[0..7] free here)
    const double hn = sqrt(red[16]);
    // Hessenberg column j, earlier rotations, new rotation, g (every CTA alike)
    if (threadIdx.x == 0) {
      double* h = H + (size_t)j * ldh;
      for (int i = 0; i <= j; ++i) h[i] = h1[i] + h2[i];
      h[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double p = h[i], q = h[i + 1];
        h[i] = cs[i] * p + sn[i] * q;
        h[i + 1] = -sn[i] * p + cs[i] * q;
      }
      const double p = h[j], q = h[j + 1];
      const double rr = hypot(p, q);
      double c = 1.0, sv = 0.0;
      if (rr != 0.0) {
        c = p / rr;
        sv = q / rr;
      }
      cs[j] = c;
      sn[j] = sv;
      h[j] = c * p + sv * q;
      h[j + 1] = 0.0;
      g[j + 1] = -sv * g[j];
      g[j] = c * g[j];
    }
    __syncthreads();
    kdone = j + 1;
    if (!(hn > 0.0) || !isfinite(hn)) {   // breakdown: the Krylov space is exhausted
      if (threadIdx.x == 0 && blockIdx.x == 0 && !isfinite(hn)) atomicOr(a.kflag, ST_NONFINITE);
      break;
    }
    inv = 1.0 / hn;
  }
  // y = H[:k,:k]^{-1} g[:k] (back substitution, into h1), x += Z y on own rows
  if (threadIdx.x == 0) {
    for (int i = kdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int c = i + 1; c < kdone; ++c) s -= H[(size_t)c * ldh + i] * h1[c];
      const double d = H[(size_t)i * ldh + i];
      h1[i] = d != 0.0 ? s / d : 0.0;
    }
  }
  __syncthreads();
  for (long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    double acc = (double)a.x[n];
    for (int i = 0; i < kdone; ++i) acc += h1[i] * (double)a.Z[(size_t)i * N + n];
    a.x[n] = (float)acc;
  }
}

static size_t coop_smem(int nu, int nb, int ld, int nf, int epc, int tpe) {
  const size_t ldh = nu + 1;
  const size_t dbl = ldh * nu + 2 * (size_t)nu + 3 * ldh + 32;
  const size_t xs = std::max((size_t)epc * (1 + nf) * nb, (size_t)(256 / tpe) * nb);
  return dbl * sizeof(double) + 4 * sizeof(int) + (xs + (size_t)epc * (1 + nf) * ld) * sizeof(float);
}

template <class S>
static cudaError_t plan_coop(int nb, int ld, int nf, int E, int nu, CoopPlan* plan) {
  constexpr int R = Col16<S>::R;
  plan->ok = 0;
  if (ld % R) return cudaSuccess;
  const int tpe = ld / R, tpb = (1 + nf) * tpe;
  if (tpb > 256 || tpe > 256) return cudaSuccess;
  const int epc = std::max(1, 256 / tpb);
  const size_t smem = coop_smem(nu, nb, ld, nf, epc, tpe);
  auto kern = coop_smooth_kernel<S>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int occ = 0, dev = 0, nsm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (occ < 1 || nsm < 1) return cudaSuccess;
  int grid = std::min(E, std::min(occ, 2) * nsm);
  const int chunk = (E + grid - 1) / grid;
  grid = (E + chunk - 1) / chunk;   // no CTA without elements
  plan->ok = 1;
  plan->nu_max = nu;
  plan->grid = grid;
  plan->chunk = chunk;
  plan->epc = epc;
  plan->tpe = tpe;
  plan->smem = smem;
  return cudaSuccess;
}

cudaError_t plan_coop_smoother(int bf16, int nb, int nf, int E, int nu, CoopPlan* plan) {
  return bf16 ? plan_coop<unsigned short>(nb, ld_bf16(nb), nf, E, nu, plan)
              : plan_coop<float>(nb, inv_ld<float>(nb), nf, E, nu, plan);
}

template <class S>
static cudaError_t launch_coop(const CoopPlan& pl, const S* Dinv, const S* Dop, const S* O, int ld, const int* nbr,
                               int nf, const float* b, float* x, int nu, Krylov<float>& K, double* part,
                               unsigned* bar, int* status, int expect_extra, int nb, int E, cudaStream_t st) {
  CoopArgs<S> a;
  a.Dinv = Dinv;
  a.Dop = Dop;
  a.O = O;
  a.nbr = nbr;
  a.b = b;
  a.x = x;
  a.V = K.V;
  a.Z = K.Z;
  a.w = K.w;
  a.part = part;
  a.bar = bar;
  a.status = status;
  a.kflag = K.kdim + 1;
  a.N = K.N;
  a.nu = nu;
  a.nb = nb;
  a.ld = ld;
  a.nf = nf;
  a.E = E;
  a.chunk = pl.chunk;
  a.epc = pl.epc;
  a.tpe = pl.tpe;
  a.expect = pl.grid + expect_extra;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, coop_smooth_kernel<S>, a);
}

cudaError_t launch_coop_smoother(const CoopPlan& pl, const float* Dinv, const float* Dop, const float* O,
                                 const unsigned short* Dinv16, const unsigned short* Dop16, const unsigned short* O16,
                                 const int* nbr, int nf, const float* b, float* x, int nu, Krylov<float>& K,
                                 double* part, unsigned* bar, int* status, int expect_extra, int nb, int E,
                                 cudaStream_t st) {
  if (!pl.ok || nu > pl.nu_max || nu > K.nmax) return cudaErrorInvalidValue;
  if (Dinv16)
    return launch_coop<unsigned short>(pl, Dinv16, Dop16, O16, ld_bf16(nb), nbr, nf, b, x, nu, K, part, bar, status,
                                       expect_extra, nb, E, st);
  return launch_coop<float>(pl, Dinv, Dop, O, inv_ld<float>(nb), nbr, nf, b, x, nu, K, part, bar, status,
                            expect_extra, nb, E, st);
}

}  // namespace dgk
