// Vector kernels and the device-resident (F)GMRES Arnoldi process (Sec. 6:
// flexible GMRES, Saad 1993; GMRES smoothers of Algorithm 2).
//
// Orthogonalisation is classical Gram-Schmidt applied twice (CGS2): the j+1
// inner products of a pass are one kernel (one CTA row per basis vector,
// fixed chunking) plus a fixed-order finalisation, so results do not depend
// on timing.  The Hessenberg column, the Givens rotations, the least-squares
// solve and the residual estimate |g_{j+1}| live in device memory; the host
// never waits on them unless it asks for the residual.
//
// FP32 vectors (the smoothers of the mixed-precision preconditioner) take
// their per-entry arithmetic in FP32 and only the sums across threads and
// CTAs in FP64: GB300 executes FP64 (and FP32<->FP64 conversions) at a small
// fraction of its FP32 rate, so a per-entry FP64 multiply-add made these
// kernels FP64-bound.  The inner products sum at most 16 FP32 products per
// thread before an FP64 add, and a CTA's threads in FP32 (one FP64 partial per
// CTA, the partials summed in FP64); the coefficients of w -= V c and x += Z y
// are rounded to FP32 once per CTA.  Classical Gram-Schmidt applied twice keeps
// the basis orthogonal to working precision with FP32 subtraction: the second
// pass removes what the rounding of the first left along V.
#include <math.h>

#include <algorithm>

#include "dg_internal.h"

namespace dgk {

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ---------------------------------------------------------------- elementwise
template <class T>
__global__ void axpby_kernel(long n, double a, const T* __restrict__ x, double b, T* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i] + (b == 0.0 ? 0.0 : b * (double)y[i]));
}
template <>
__global__ void axpby_kernel<float>(long n, double a, const float* __restrict__ x, double b, float* __restrict__ y) {
  float af = (float)a, bf = (float)b;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = af * x[i] + (b == 0.0 ? 0.0f : bf * y[i]);
}

static int grid_for(long n) {
  long g = (n + 255) / 256;
  return (int)std::max<long>(1, std::min<long>(g, 8L * sm_count()));
}

template <class T>
cudaError_t launch_axpby(long n, double a, const T* x, double b, T* y, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  axpby_kernel<T><<<grid_for(n), 256, 0, st>>>(n, a, x, b, y);
  return cudaGetLastError();
}
template cudaError_t launch_axpby<double>(long, double, const double*, double, double*, cudaStream_t);
template cudaError_t launch_axpby<float>(long, double, const float*, double, float*, cudaStream_t);

template <class A, class B>
__global__ void convert_kernel(long n, const A* __restrict__ x, B* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = (B)x[i];
}
template <class A, class B>
cudaError_t launch_convert(long n, const A* x, B* y, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  convert_kernel<A, B><<<grid_for(n), 256, 0, st>>>(n, x, y);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(long, const double*, float*, cudaStream_t);
template cudaError_t launch_convert<float, double>(long, const float*, double*, cudaStream_t);

// restriction I_l^{l+1}: keep the leading modes of every (element, variable)
template <class T>
__global__ void restrict_kernel(const T* __restrict__ xf, int nmf, T* __restrict__ xc, int nmc, long nev) {
  long tot = nev * nmc;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    long ev = t / nmc;
    int i = (int)(t % nmc);
    xc[t] = xf[ev * nmf + i];
  }
}
// prolongation I_{l+1}^l = (I_l^{l+1})^T: zero-pad (add = false) or add into xf
template <class T>
__global__ void prolong_kernel(const T* __restrict__ xc, int nmc, T* __restrict__ xf, int nmf, long nev, int add) {
  long tot = nev * nmf;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    long ev = t / nmf;
    int i = (int)(t % nmf);
    T c = i < nmc ? xc[ev * nmc + i] : T(0);
    xf[t] = add ? xf[t] + c : c;
  }
}
template <class T>
cudaError_t launch_restrict(const T* xf, int nmf, T* xc, int nmc, long nev, cudaStream_t st) {
  note_launch();
  restrict_kernel<T><<<grid_for(nev * nmc), 256, 0, st>>>(xf, nmf, xc, nmc, nev);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_prolong(const T* xc, int nmc, T* xf, int nmf, long nev, bool add, cudaStream_t st) {
  note_launch();
  prolong_kernel<T><<<grid_for(nev * nmf), 256, 0, st>>>(xc, nmc, xf, nmf, nev, add ? 1 : 0);
  return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const double*, int, double*, int, long, cudaStream_t);
template cudaError_t launch_restrict<float>(const float*, int, float*, int, long, cudaStream_t);
template cudaError_t launch_prolong<double>(const double*, int, double*, int, long, bool, cudaStream_t);
template cudaError_t launch_prolong<float>(const float*, int, float*, int, long, bool, cudaStream_t);

// ---------------------------------------------------------------- reductions
// part[i][c] = sum over chunk c of V_i . w (FP64 accumulation), i < nvec.
template <class T>
__global__ void __launch_bounds__(256) mdot_kernel(const T* __restrict__ V, long N, const T* __restrict__ w,
                                                   int G, double* __restrict__ part) {
  __shared__ double red[256];
  const int i = blockIdx.y, c = blockIdx.x;
  const long chunk = (N + G - 1) / G;
  const long beg = c * chunk, end = min(N, beg + chunk);
  const T* v = V + (size_t)i * N;
  double s = 0.0;
  for (long n = beg + threadIdx.x; n < end; n += blockDim.x) s += (double)v[n] * (double)w[n];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)i * G + c] = red[0];
}
template <>
__global__ void __launch_bounds__(256) mdot_kernel<float>(const float* __restrict__ V, long N,
                                                          const float* __restrict__ w, int G,
                                                          double* __restrict__ part) {
  // the CTA's sum in FP32 (a thread's products 16 at a time into FP64, then warp
  // butterflies and the eight warp sums in FP32: FP64 adds have long latencies
  // here), one FP64 partial per CTA; the CTAs' partials are summed in FP64
  __shared__ float red[8];
  const int i = blockIdx.y, c = blockIdx.x;
  const long chunk = (N + G - 1) / G;
  const long beg = c * chunk, end = min(N, beg + chunk);
  const float* v = V + (size_t)i * N;
  double s = 0.0;
  for (long n0 = beg + threadIdx.x; n0 < end; n0 += 16L * blockDim.x) {
    float f = 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const long n = n0 + (long)u * blockDim.x;
      if (n < end) f = fmaf(v[n], w[n], f);
    }
    s += (double)f;
  }
  float t = (float)s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b += red[k];
    part[(size_t)i * G + c] = (double)b;
  }
}

// mode 0: H[i][j] = sum; mode 1: H[i][j] += sum;  (one warp per i, fixed order)
__global__ void finalize_dots_kernel(const double* __restrict__ part, int G, int nvec, double* __restrict__ Hcol,
                                     double* __restrict__ tmp, int mode) {
  int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (i >= nvec) return;
  double s = 0.0;
  for (int c = lane; c < G; c += 32) s += part[(size_t)i * G + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    if (mode == 0) Hcol[i] = s;
    else {
      tmp[i] = s;
      Hcol[i] += s;
    }
  }
}

// w -= sum_i c[i] V_i, c read from device memory
template <class T>
__global__ void subtract_kernel(const T* __restrict__ V, long N, const double* __restrict__ c, int nvec,
                                T* __restrict__ w) {
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
    double acc = (double)w[n];
    for (int i = 0; i < nvec; ++i) acc -= c[i] * (double)V[(size_t)i * N + n];
    w[n] = (T)acc;
  }
}
// FP32: the coefficients rounded once into shared memory (nvec <= KMAX_F32)
constexpr int KMAX_F32 = 128;
template <>
__global__ void subtract_kernel<float>(const float* __restrict__ V, long N, const double* __restrict__ c, int nvec,
                                       float* __restrict__ w) {
  __shared__ float cf[KMAX_F32];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) cf[i] = (float)c[i];
  __syncthreads();
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
    float acc = w[n];
    for (int i = 0; i < nvec; ++i) acc = fmaf(-cf[i], V[(size_t)i * N + n], acc);
    w[n] = acc;
  }
}

// norm finalisation: nrm = sqrt(sum part[0..G)); writes *dst = nrm, *inv = 1/nrm
// (0 when nrm == 0, with kdim lowered to `brk`), and for start(): g = (nrm, 0...).
__global__ void finalize_norm_kernel(const double* __restrict__ part, int G, double* dst, double* inv, int* kdim,
                                     int brk, double* g, int gN, int* status) {
  int lane = threadIdx.x;
  double s = 0.0;
  for (int c = lane; c < G; c += 32) s += part[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double nrm = sqrt(s);
    if (!isfinite(nrm)) {
      atomicOr(status, ST_NONFINITE);
      nrm = 0.0;
    }
    *dst = nrm;
    *inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (!(nrm > 0.0) && *kdim > brk) *kdim = brk;
    if (g) {
      g[0] = nrm;
      for (int t = 1; t < gN; ++t) g[t] = 0.0;
    }
  }
}

template <class T>
__global__ void scale_kernel(long N, const T* __restrict__ x, const double* __restrict__ inv, T* __restrict__ y) {
  double a = *inv;
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x)
    y[n] = (T)(a * (double)x[n]);
}
template <>
__global__ void scale_kernel<float>(long N, const float* __restrict__ x, const double* __restrict__ inv,
                                    float* __restrict__ y) {
  const float a = (float)*inv;
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x)
    y[n] = a * x[n];
}

// Givens update of Hessenberg column j (column-major, ld = nmax+1).
__global__ void givens_kernel(double* H, int ld, double* cs, double* sn, double* g, int j, double* res) {
  if (threadIdx.x != 0) return;
  double* h = H + (size_t)j * ld;
  for (int i = 0; i < j; ++i) {
    double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  double a = h[j], b = h[j + 1];
  double r = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (r != 0.0) {
    c = a / r;
    s = b / r;
  }
  cs[j] = c;
  sn[j] = s;
  h[j] = c * a + s * b;
  h[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  *res = fabs(g[j + 1]);
}

// y = H[:k,:k]^{-1} g[:k], k = min(kdone, kdim)
__global__ void lsq_kernel(const double* H, int ld, const double* g, int kdone, const int* kdim, double* y,
                           int nmax) {
  if (threadIdx.x != 0) return;
  int k = min(kdone, *kdim);
  for (int i = 0; i < nmax; ++i) y[i] = 0.0;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(size_t)c * ld + i] * y[c];
    double d = H[(size_t)i * ld + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// x += Z y over the first min(k, *kdim) directions (the directions past the
// effective Krylov dimension may hold anything: they are not read)
template <class T>
__global__ void update_kernel(const T* __restrict__ Z, long N, const double* __restrict__ y, int k,
                              const int* __restrict__ kdim, T* __restrict__ x) {
  k = min(k, *kdim);
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
    double acc = (double)x[n];
    for (int i = 0; i < k; ++i) acc += y[i] * (double)Z[(size_t)i * N + n];
    x[n] = (T)acc;
  }
}
template <>
__global__ void update_kernel<float>(const float* __restrict__ Z, long N, const double* __restrict__ y, int k,
                                     const int* __restrict__ kdim, float* __restrict__ x) {
  __shared__ float yf[KMAX_F32];
  k = min(k, *kdim);
  for (int i = threadIdx.x; i < k; i += blockDim.x) yf[i] = (float)y[i];
  __syncthreads();
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
    float acc = x[n];
    for (int i = 0; i < k; ++i) acc = fmaf(yf[i], Z[(size_t)i * N + n], acc);
    x[n] = acc;
  }
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

// ---------------------------------------------------------------- Krylov
template <class T>
cudaError_t Krylov<T>::alloc(long n, int nm) {
  release();
  if (sizeof(T) == sizeof(float) && nm + 1 > KMAX_F32) return cudaErrorInvalidValue;
  N = n;
  nmax = nm;
  G = (int)std::max<long>(1, std::min<long>(2L * sm_count(), (n + 1023) / 1024));
  auto get = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 8));
    if (e == cudaSuccess) allocs.push_back(*p);
    return e;
  };
  cudaError_t e;
  if ((e = get((void**)&V, sizeof(T) * (size_t)(nm + 1) * n))) return e;
  if ((e = get((void**)&Z, sizeof(T) * (size_t)nm * n))) return e;
  if ((e = get((void**)&w, sizeof(T) * (size_t)n))) return e;
  if ((e = get((void**)&H, sizeof(double) * (size_t)(nm + 1) * nm))) return e;
  if ((e = get((void**)&cs, sizeof(double) * nm))) return e;
  if ((e = get((void**)&sn, sizeof(double) * nm))) return e;
  if ((e = get((void**)&g, sizeof(double) * (nm + 1)))) return e;
  if ((e = get((void**)&y, sizeof(double) * (nm + 2)))) return e;
  if ((e = get((void**)&part, sizeof(double) * (size_t)(nm + 2) * G))) return e;
  if ((e = get((void**)&res, sizeof(double) * 4))) return e;
  if ((e = get((void**)&kdim, sizeof(int) * 2))) return e;
  if ((e = cudaMemset(kdim, 0, sizeof(int) * 2))) return e;
  return cudaMemset(H, 0, sizeof(double) * (size_t)(nm + 1) * nm);
}

template <class T>
void Krylov<T>::release() {
  for (void* p : allocs) cudaFree(p);
  allocs.clear();
  V = Z = w = nullptr;
  H = cs = sn = g = y = part = res = nullptr;
  kdim = nullptr;
}

template <class T>
size_t Krylov<T>::bytes() const {
  return sizeof(T) * (size_t)(2 * nmax + 2) * N;
}

template <class T>
static cudaError_t norm_into(const Krylov<T>& K, const T* x, double* dst, double* inv, int brk, double* g,
                             int gN, cudaStream_t st) {
  dim3 grid(K.G, 1);
  note_launch();
  mdot_kernel<T><<<grid, 256, 0, st>>>(x, K.N, x, K.G, K.part);
  note_launch();
  finalize_norm_kernel<<<1, 32, 0, st>>>(K.part, K.G, dst, inv, K.kdim, brk, g, gN, K.kdim + 1);
  return cudaGetLastError();
}

template <class T>
cudaError_t Krylov<T>::start(const T* r, cudaStream_t st) {
  note_launch();
  set_int_kernel<<<1, 1, 0, st>>>(kdim, nmax);
  cudaError_t e = norm_into(*this, r, res + 1, res + 2, 0, g, nmax + 1, st);
  if (e) return e;
  note_launch();
  scale_kernel<T><<<grid_for(N), 256, 0, st>>>(N, r, res + 2, V);
  return cudaGetLastError();
}

template <class T>
cudaError_t Krylov<T>::arnoldi(int j, cudaStream_t st) {
  const int nv = j + 1;
  double* Hcol = H + (size_t)j * (nmax + 1);
  int fgrid = (nv + 7) / 8;
  for (int pass = 0; pass < 2; ++pass) {
    dim3 grid(G, nv);
    note_launch();
    mdot_kernel<T><<<grid, 256, 0, st>>>(V, N, w, G, part);
    note_launch();
    finalize_dots_kernel<<<fgrid, 256, 0, st>>>(part, G, nv, Hcol, y, pass);
    // pass 0 subtracts H[:,j] (h1), pass 1 subtracts the correction h2 (kept in y)
    note_launch();
    subtract_kernel<T><<<grid_for(N), 256, 0, st>>>(V, N, pass == 0 ? Hcol : y, nv, w);
  }
  cudaError_t e = norm_into(*this, w, Hcol + j + 1, res + 2, j + 1, nullptr, 0, st);
  if (e) return e;
  note_launch();
  scale_kernel<T><<<grid_for(N), 256, 0, st>>>(N, w, res + 2, V + (size_t)(j + 1) * N);
  note_launch();
  givens_kernel<<<1, 32, 0, st>>>(H, nmax + 1, cs, sn, g, j, res);
  return cudaGetLastError();
}

template <class T>
cudaError_t Krylov<T>::update(int kdone, T* x, cudaStream_t st) {
  note_launch();
  lsq_kernel<<<1, 32, 0, st>>>(H, nmax + 1, g, kdone, kdim, y, nmax);
  note_launch();
  update_kernel<T><<<grid_for(N), 256, 0, st>>>(Z, N, y, kdone, kdim, x);
  return cudaGetLastError();
}

template struct Krylov<double>;
template struct Krylov<float>;

}  // namespace dgk
