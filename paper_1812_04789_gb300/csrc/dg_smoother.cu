// Persistent GMRES(BJ) smoother of the inherited coarse levels: one
// cooperative launch runs a whole SMOOTH / SOLVE call of Algorithm 2 (nu
// iterations of GMRES right-preconditioned by element block Jacobi, Sec. 6.3,
// on the inherited block-sparse operator of Sec. 6.1), where the
// launch-per-operation path takes about eleven small kernels per iteration.
//
// One CTA per SM owns a contiguous range of elements for the whole call and
// keeps its rows of the Krylov basis V, of the preconditioned directions Z and
// of the work vector w in shared memory (the coarse levels are small: a level
// whose rows do not fit keeps the launch-per-operation smoother).  Only z_j
// goes to device memory, where the neighbours' products read it.  Per
// iteration j:
//   A  v_j = w / ||w||; z_j = D^{-1} v_j (own elements)                 | grid barrier
//   B  w = A z_j (own elements, neighbours' z_j read); partial V^T w    | grid barrier
//   C  h1 = sum of partials; w -= V h1; partial V^T w and ||w||^2       | grid barrier
//   D  h2 = sum of partials; w -= V h2; ||w - V h2||^2 = ||w||^2 - ||h2||^2
// (CGS2, as the launch-per-operation Arnoldi; the norm after the second pass
// by Pythagoras, as in the low-synchronisation Gram-Schmidt variants of
// Swirydowicz et al. 2021, which saves a barrier: h2 is at rounding level
// against w, so the difference loses nothing.  Where it would cancel, more
// than 99 % of ||w||^2, the norm is summed explicitly behind a fourth
// barrier; every CTA takes the same branch.)  A barrier that ends a
// reduction also sums it: the last CTA to arrive adds the CTAs' partials in a
// fixed order (FP64) and publishes the sums before it releases the others,
// which then read only the sums.  Every CTA keeps its own copy of the
// Hessenberg matrix, the Givens rotations and g, so all CTAs hold identical
// scalars and the final x += Z y needs no further barrier.  The arithmetic
// inside a CTA is FP32 (products and their sums over the CTA's rows, w -= V h
// with h rounded to FP32, the Givens rotations and the small least-squares
// solve, x += Z y): GB300 runs FP64 and FP32<->FP64 conversions at a small
// fraction of its FP32 rate, with long latencies, and FP64 there made the
// smoother FP64-bound; only the sums across CTAs are FP64.
//
// The grid barrier counts arrivals in one word and releases the waiting CTAs
// through another (its own 128-byte line, so the polls do not contend with
// the arrivals); both are zeroed before the launch.  Every wait is bounded
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
  float* Z;             // nu x N: the directions z_j, read by the neighbours' products
  double* part;         // [grid][2 (nu + 1) + 1] partials, then one row of sums
  unsigned* bar;        // [0]: arrivals, [32]: released barrier number; zero at launch
  int* status;          // mesh status word (ST_TIMEOUT)
  int* kflag;           // Krylov status bits (ST_NONFINITE)
  long N;
  int nu, nb, ld, nf, E, chunk, epc, tpe, expect;
};

constexpr int COOP_THREADS = 512;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier number k (k * expect arrivals); false when a wait ran out
// here or elsewhere (ST_TIMEOUT), and then the caller returns.
__device__ bool grid_barrier(unsigned* bar, unsigned k, unsigned expect, int* status, int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned old = atomicAdd(bar, 1u);
    if (old + 1u == k * expect) {
      __threadfence();
      atomicExch(bar + 32, k);            // the last arrival releases barrier k
    } else {
      const unsigned long long t0 = global_ns();
      while (*(volatile unsigned*)(bar + 32) < k) {
        if (*(volatile int*)status & ST_TIMEOUT) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > 2000000000ull) {
          atomicOr(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// Grid barrier number k that also sums the CTAs' partials: the last CTA to
// arrive adds part[c * stride + off + i] over c = 0..G-1 for i < nv (16 lanes
// per value, each lane its c = lane, lane + 16, .. loaded at once and summed as
// a tree, then a butterfly: the same order whichever CTA is last) into tot[i], then releases the
// others; every CTA copies tot[0, nv) into dst (shared memory).  One CTA reads
// the G x nv partials instead of every CTA.  False when a wait ran out here or
// elsewhere (ST_TIMEOUT), and then the caller returns.
__device__ bool grid_barrier_sum(unsigned* bar, unsigned k, unsigned expect, int* status, int* sflag,
                                 const double* part, int stride, int off, int nv, int G, double* tot,
                                 double* dst) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(bar, 1u);
    __threadfence();
    sflag[2] = old + 1u == k * expect ? 1 : 0;
  }
  __syncthreads();
  if (sflag[2]) {
    const int grp = threadIdx.x >> 4, l16 = threadIdx.x & 15, ngrp = blockDim.x >> 4;
    for (int i0 = 0; i0 < nv; i0 += ngrp) {
      const int i = i0 + grp;   // uniform per 16-lane group
      // every load of a lane issued at once (12 per lane: G <= 192 in one
      // round trip), summed as a tree
      double t[12];
#pragma unroll
      for (int u = 0; u < 12; ++u) {
        const int c = l16 + 16 * u;
        t[u] = (i < nv && c < G) ? __ldcg(part + (size_t)c * stride + off + i) : 0.0;
      }
      double s = (((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]))) +
                 ((t[8] + t[9]) + (t[10] + t[11]));
      for (int c = l16 + 192; i < nv && c < G; c += 16) s += __ldcg(part + (size_t)c * stride + off + i);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (i < nv && l16 == 0) tot[i] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicExch(bar + 32, k);            // release barrier k
      sflag[0] = 1;
    }
  } else if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long t0 = global_ns();
    while (*(volatile unsigned*)(bar + 32) < k) {
      if (*(volatile int*)status & ST_TIMEOUT) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > 2000000000ull) {
        atomicOr(status, ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
    sflag[0] = ok;
  }
  __syncthreads();
  if (!sflag[0]) return false;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = __ldcg(tot + i);
  __syncthreads();
  return true;
}

// FP32 sum over the CTA's threads of f (warp butterflies, then warp 0 over
// the warp sums), valid in every thread; redf: 33 floats, [32] the result
__device__ float block_sum_f(float f, float* redf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();   // earlier readers of redf are done
  if (lane == 0) redf[warp] = f;
  __syncthreads();
  if (warp == 0) {
    float t = lane < nw ? redf[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) redf[32] = t;
  }
  __syncthreads();
  return redf[32];
}

// out[i] = sum over the CTA's rows of V_i . w (shared memory), i < nv, warp per
// i, in FP32 (a lane's rows, then the warp's butterfly); the CTA partials are
// then summed across CTAs in FP64
__device__ void own_dots(int nv, const float* Vs, int ldv, const float* ws, int rows, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < nv; i += nw) {
    const float* v = Vs + (size_t)i * ldv;
    float f0 = 0.f, f1 = 0.f;
    int r = lane;
    for (; r + 32 < rows; r += 64) {
      f0 = fmaf(v[r], ws[r], f0);
      f1 = fmaf(v[r + 32], ws[r + 32], f1);
    }
    if (r < rows) f0 = fmaf(v[r], ws[r], f0);
    float f = f0 + f1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) out[i] = (double)f;
  }
}

// ws[own rows of e] = [b_e -] (D_e in_e + sum_s O_{e,s} in_nbr(e,s)) for the
// CTA's ne elements from e_beg: a thread per (element, R rows) sums all the
// element's blocks, column by column with the 1 + NF blocks' loads of a column
// in flight together (the coarse levels are latency-bound); the inputs are
// staged in shared memory, epc elements a pass.
template <class S, int NF>
__device__ void bsr_own(const CoopArgs<S>& a, const float* in, const float* bsub, float* ws, int e_beg, int ne,
                        float* xs) {
  constexpr int R = Col16<S>::R, NSRC = 1 + NF;
  const int nb = a.nb, ld = a.ld, tpe = a.tpe, epc = a.epc;
  const size_t bs = (size_t)nb * ld;
  const int sub = threadIdx.x / tpe, tt = threadIdx.x - sub * tpe;
  for (int p0 = 0; p0 < ne; p0 += epc) {
    const int nl = min(epc, ne - p0);
    for (int t = threadIdx.x; t < nl * NSRC * nb; t += blockDim.x) {
      const int el = t / (NSRC * nb), q = t - el * NSRC * nb, who = q / nb, j = q - who * nb;
      const int e = e_beg + p0 + el;
      const int src = who == 0 ? e : a.nbr[(size_t)e * NF + who - 1];
      xs[t] = __ldcg(in + (size_t)src * nb + j);
    }
    __syncthreads();
    if (sub < nl) {
      const int e = e_beg + p0 + sub;
      const S* base[NSRC];
      base[0] = a.Dop + (size_t)e * bs + R * tt;
#pragma unroll
      for (int b = 1; b < NSRC; ++b) base[b] = a.O + ((size_t)e * NF + b - 1) * bs + R * tt;
      const float* xe = xs + (size_t)sub * NSRC * nb;
      float acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = 0.f;
#pragma unroll 2
      for (int c = 0; c < nb; ++c) {
        float v[NSRC][R];
#pragma unroll
        for (int b = 0; b < NSRC; ++b) Col16<S>::load(base[b] + (size_t)c * ld, v[b]);
#pragma unroll
        for (int b = 0; b < NSRC; ++b) {
          const float xv = xe[(size_t)b * nb + c];
#pragma unroll
          for (int j = 0; j < R; ++j) acc[j] += v[b][j] * xv;
        }
      }
      const int r0 = (p0 + sub) * nb + R * tt;
      const size_t n0 = (size_t)e_beg * nb;
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (R * tt + j < nb) ws[r0 + j] = bsub ? __ldcg(bsub + n0 + r0 + j) - acc[j] : acc[j];
    }
    __syncthreads();
  }
}

// z_e = D_e^{-1} v_e for the CTA's elements: v from shared memory, z to shared
// memory (own rows) and device memory (the neighbours' products read it)
template <class S>
__device__ void bj_own(const CoopArgs<S>& a, const float* vs, float* zs, float* zg, int e_beg, int ne) {
  constexpr int R = Col16<S>::R;
  const int nb = a.nb, ld = a.ld, tpe = a.tpe, epc = blockDim.x / tpe;
  const size_t bs = (size_t)nb * ld;
  const int sub = threadIdx.x / tpe, tt = threadIdx.x - sub * tpe;
  for (int p0 = 0; p0 < ne; p0 += epc) {
    const int nl = min(epc, ne - p0);
    if (sub < nl) {
      const S* base = a.Dinv + (size_t)(e_beg + p0 + sub) * bs + R * tt;
      const float* xe = vs + (size_t)(p0 + sub) * nb;
      float acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = 0.f;
#pragma unroll 16
      for (int c = 0; c < nb; ++c) {
        float m[R];
        Col16<S>::load(base + (size_t)c * ld, m);
        const float xv = xe[c];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += m[j] * xv;
      }
      const int r0 = (p0 + sub) * nb + R * tt;
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (R * tt + j < nb) {
          zs[r0 + j] = acc[j];
          zg[(size_t)e_beg * nb + r0 + j] = acc[j];
        }
    }
  }
}

template <class S, int NF>
__global__ void __launch_bounds__(COOP_THREADS, 1) coop_smooth_kernel(CoopArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nu = a.nu, ldh = nu + 1, nb = a.nb;
  double* h1 = reinterpret_cast<double*>(smem_raw);   // nu + 1: first-pass coefficients (FP64 sums)
  double* h2 = h1 + ldh;                              // nu + 2: second pass, then ||w||^2
  double* hx = h2 + ldh + 1;                          // 2: broadcast scalars
  int* sflag = reinterpret_cast<int*>(hx + 2);        // 4 ints
  float* H = reinterpret_cast<float*>(sflag + 4);     // (nu + 1) x nu, column-major
  float* cs = H + (size_t)ldh * nu;
  float* sn = cs + nu;
  float* g = sn + nu;                                 // nu + 1
  float* hf = g + ldh;                                // nu + 1: coefficients rounded to FP32, then y
  float* redf = hf + ldh;                             // 33
  const int rmax = a.chunk * nb;
  float* Vs = redf + ((33 + 3) & ~3);                 // [nu + 1][rmax]
  float* Zs = Vs + (size_t)ldh * rmax;                // [nu][rmax]
  float* ws = Zs + (size_t)nu * rmax;                 // [rmax]
  float* xs = ws + rmax;                              // [epc][1 + nf][nb]

  const int G = gridDim.x, stride = 2 * ldh + 1;
  double* mypart = a.part + (size_t)blockIdx.x * stride;   // [0, ldh): pass 1, [ldh, 2 ldh): pass 2, last: norm
  double* tot = a.part + (size_t)G * stride;               // the sums, written by the last CTA of a barrier
  const int e_beg = min(a.E, (int)blockIdx.x * a.chunk), ne = min(a.E, e_beg + a.chunk) - e_beg;
  const int rows = ne * nb;
  const long N = a.N;
  const unsigned expect = (unsigned)a.expect;
  unsigned nbar = 0;

  if (threadIdx.x == 0) sflag[1] = (*(volatile int*)a.status & ST_TIMEOUT) ? 1 : 0;
  __syncthreads();
  if (sflag[1]) return;   // an earlier wait ran out: leave x as it is

  // r = b - A x into w, ||r||^2
  bsr_own<S, NF>(a, a.x, a.b, ws, e_beg, ne, xs);
  {
    float f = 0.f;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) f = fmaf(ws[r], ws[r], f);
    const float s = block_sum_f(f, redf);
    if (threadIdx.x == 0) mypart[2 * ldh] = (double)s;
  }
  if (!grid_barrier_sum(a.bar, ++nbar, expect, a.status, sflag, a.part, stride, 2 * ldh, 1, G, tot, h2)) return;
  const double beta = sqrt(h2[0]);
  if (!(beta > 0.0) || !isfinite(beta)) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !isfinite(beta)) atomicOr(a.kflag, ST_NONFINITE);
    return;   // b - A x = 0 (or not finite): nothing to smooth
  }
  for (int i = threadIdx.x; i < ldh; i += blockDim.x) g[i] = i == 0 ? (float)beta : 0.f;
  float finv = (float)(1.0 / beta);
  int kdone = 0;
  for (int j = 0; j < nu; ++j) {
    // A: v_j = w / ||w||, z_j = D^{-1} v_j
    float* vj = Vs + (size_t)j * rmax;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) vj[r] = finv * ws[r];
    __syncthreads();
    float* zg = a.Z + (size_t)j * N;
    bj_own<S>(a, vj, Zs + (size_t)j * rmax, zg, e_beg, ne);
    if (!grid_barrier(a.bar, ++nbar, expect, a.status, sflag)) return;
    // B: w = A z_j, first pass of inner products
    bsr_own<S, NF>(a, zg, nullptr, ws, e_beg, ne, xs);
    own_dots(j + 1, Vs, rmax, ws, rows, mypart);
    if (!grid_barrier_sum(a.bar, ++nbar, expect, a.status, sflag, a.part, stride, 0, j + 1, G, tot, h1)) return;
    // C: w -= V h1; second pass of inner products and ||w||^2 (at mypart[ldh + j + 1])
    if (threadIdx.x <= j) hf[threadIdx.x] = (float)h1[threadIdx.x];
    __syncthreads();
    {
      float f = 0.f;
      for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        float acc = ws[r];
        for (int i = 0; i <= j; ++i) acc = fmaf(-hf[i], Vs[(size_t)i * rmax + r], acc);
        ws[r] = acc;
        f = fmaf(acc, acc, f);
      }
      const float s = block_sum_f(f, redf);
      own_dots(j + 1, Vs, rmax, ws, rows, mypart + ldh);
      if (threadIdx.x == 0) mypart[ldh + j + 1] = (double)s;
    }
    if (!grid_barrier_sum(a.bar, ++nbar, expect, a.status, sflag, a.part, stride, ldh, j + 2, G, tot, h2))
      return;   // h2[j + 1] = ||w||^2
    // D: w -= V h2, ||w - V h2|| from ||w||^2 - ||h2||^2; Hessenberg column j
    // (h1 + h2, formed in parallel) in FP32
    if (threadIdx.x <= j) {
      hf[threadIdx.x] = (float)h2[threadIdx.x];
      H[(size_t)j * ldh + threadIdx.x] = (float)(h1[threadIdx.x] + h2[threadIdx.x]);
    }
    if (threadIdx.x < 32) {   // ||h2||^2 (FP32: h2 is at rounding level against ||w||)
      float q = 0.f;
      for (int i = threadIdx.x; i <= j; i += 32) {
        const float t = (float)h2[i];
        q = fmaf(t, t, q);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if (threadIdx.x == 0) hx[0] = h2[j + 1] - (double)q;
    }
    __syncthreads();
    const double nw2 = h2[j + 1], hn2 = hx[0];
    const bool explicit_norm = !(hn2 >= 0.01 * nw2);   // cancellation (or not finite): sum it
    {
      float f = 0.f;
      for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        float acc = ws[r];
        for (int i = 0; i <= j; ++i) acc = fmaf(-hf[i], Vs[(size_t)i * rmax + r], acc);
        ws[r] = acc;
        f = fmaf(acc, acc, f);
      }
      if (explicit_norm) {
        const float s = block_sum_f(f, redf);
        if (threadIdx.x == 0) mypart[2 * ldh] = (double)s;
      }
    }
    double hn;
    if (explicit_norm) {
      if (!grid_barrier_sum(a.bar, ++nbar, expect, a.status, sflag, a.part, stride, 2 * ldh, 1, G, tot, hx + 1))
        return;
      hn = sqrt(hx[1]);
    } else {
      hn = sqrt(hn2);
    }
    // earlier rotations, new rotation, g (every CTA alike, FP32)
    if (threadIdx.x == 0) {
      float* h = H + (size_t)j * ldh;
      h[j + 1] = (float)hn;
      for (int i = 0; i < j; ++i) {
        const float p = h[i], q = h[i + 1];
        h[i] = cs[i] * p + sn[i] * q;
        h[i + 1] = -sn[i] * p + cs[i] * q;
      }
      const float p = h[j], q = h[j + 1];
      const float rr = hypotf(p, q);
      float c = 1.f, sv = 0.f;
      if (rr != 0.f) {
        c = p / rr;
        sv = q / rr;
      }
      cs[j] = c;
      sn[j] = sv;
      h[j] = c * p + sv * q;
      h[j + 1] = 0.f;
      g[j + 1] = -sv * g[j];
      g[j] = c * g[j];
    }
    __syncthreads();
    kdone = j + 1;
    if (!(hn > 0.0) || !isfinite(hn)) {   // breakdown: the Krylov space is exhausted
      if (threadIdx.x == 0 && blockIdx.x == 0 && !isfinite(hn)) atomicOr(a.kflag, ST_NONFINITE);
      break;
    }
    finv = (float)(1.0 / hn);
  }
  // y = H[:k,:k]^{-1} g[:k] (back substitution, FP32, into hf), x += Z y on own rows
  if (threadIdx.x == 0) {
    for (int i = kdone - 1; i >= 0; --i) {
      float s = g[i];
      for (int c = i + 1; c < kdone; ++c) s -= H[(size_t)c * ldh + i] * hf[c];
      const float d = H[(size_t)i * ldh + i];
      hf[i] = d != 0.f ? s / d : 0.f;
    }
  }
  __syncthreads();
  float* xo = a.x + (size_t)e_beg * nb;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    float acc = xo[r];
    for (int i = 0; i < kdone; ++i) acc = fmaf(hf[i], Zs[(size_t)i * rmax + r], acc);
    xo[r] = acc;
  }
}

static size_t coop_smem(int nu, int nb, int nf, int chunk, int epc) {
  const size_t ldh = nu + 1;
  const size_t dbl = 2 * ldh + 1 + 2;
  const size_t fsc = ldh * nu + 2 * (size_t)nu + 2 * ldh + 36;   // H, cs, sn, g, hf, redf (padded)
  const size_t rmax = (size_t)chunk * nb;
  const size_t flt = (2 * (size_t)nu + 2) * rmax + (size_t)epc * (1 + nf) * nb;
  return dbl * sizeof(double) + 4 * sizeof(int) + (fsc + flt) * sizeof(float) + 16;
}

template <class S, int NF>
static cudaError_t plan_coop(int nb, int ld, int nf, int E, int nu, CoopPlan* plan) {
  constexpr int R = Col16<S>::R;
  plan->ok = 0;
  if (ld % R || E < 1) return cudaSuccess;
  const int tpe = ld / R;
  if (tpe > COOP_THREADS) return cudaSuccess;
  auto kern = coop_smooth_kernel<S, NF>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (nsm < 1) return cudaSuccess;
  int grid = std::min(E, nsm);
  const int chunk = (E + grid - 1) / grid;
  grid = (E + chunk - 1) / chunk;   // no CTA without elements
  const int epc = std::max(1, std::min(chunk, COOP_THREADS / tpe));
  const size_t smem = coop_smem(nu, nb, nf, chunk, epc);
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (smem + fa.sharedSizeBytes > (size_t)smax) return cudaSuccess;   // the rows do not fit: per-operation smoother
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, COOP_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaSuccess;
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
  plan->ok = 0;
  if (nf == 6)
    return bf16 ? plan_coop<unsigned short, 6>(nb, ld_bf16(nb), nf, E, nu, plan)
                : plan_coop<float, 6>(nb, inv_ld<float>(nb), nf, E, nu, plan);
  if (nf == 4)
    return bf16 ? plan_coop<unsigned short, 4>(nb, ld_bf16(nb), nf, E, nu, plan)
                : plan_coop<float, 4>(nb, inv_ld<float>(nb), nf, E, nu, plan);
  return cudaSuccess;   // other face counts keep the launch-per-operation smoother
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
  a.Z = K.Z;
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
  cudaError_t e = cudaMemsetAsync(bar, 0, COOP_BAR_WORDS * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.grid);
  cfg.blockDim = dim3(COOP_THREADS);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  if (nf == 6) return cudaLaunchKernelEx(&cfg, coop_smooth_kernel<S, 6>, a);
  return cudaLaunchKernelEx(&cfg, coop_smooth_kernel<S, 4>, a);
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
