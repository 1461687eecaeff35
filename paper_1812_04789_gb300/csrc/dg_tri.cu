// Triangular meshes: periodic triangulations with general edge connectivity,
// the full-order space P_p on every triangle (Sec. 3: polynomials of total
// degree <= k on triangular grids; Sec. 7.2: a quadrilateral grid split into
// triangles), residual and exact JVP of Sec. 3.1 eq. dg_ns with per-triangle
// affine geometry.
//
// Reference triangle {r, s >= -1, r + s <= 0}, vertices (-1,-1), (1,-1),
// (-1,1); local edges v0->v1, v1->v2, v2->v0.  Basis: orthonormal Dubiner
// polynomials sqrt(2) Ph_i(a) Ph_j^(2i+1,0)(b) (1-b)^i, a = 2(1+r)/(1-s) - 1,
// b = s (Ph: unit-norm Jacobi polynomials), ordered by total degree i + j,
// then i descending; reference derivatives by the complex step.  Volume rule:
// collapsed Gauss-Legendre, nq1d^2 points; edges: nq1d Gauss-Legendre points
// in the edge's direction (the neighbour sees them in reverse order).
//
// Each triangle evaluates its own three edges (tri_face_kernel writes one
// face slot per (triangle, edge)); tri_volume_kernel adds the volume term,
// the three slots and sigma |J| V (JVP) or -S.  The BR2 lifting of one edge
// acts through P_f[q][q'] = sum_i phi_i(q) phi_i(q') of that edge (eq. re with
// the mass matrix |J| I of the orthonormal basis).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <map>
#include <tuple>
#include <type_traits>
#include <vector>

#include "dg_internal.h"

namespace dgk {

// ---------------------------------------------------------------- host tables
namespace {

template <class C>
void jacobi_all(int n, double alpha, C x, std::vector<C>& P) {
  P.assign(n + 1, C(0.0));
  P[0] = C(1.0);
  if (n >= 1) P[1] = ((alpha + 2.0) * x + alpha) / 2.0;
  for (int k = 1; k < n; ++k) {
    const double c = 2.0 * k + alpha;
    P[k + 1] = ((c + 1.0) * ((c + 2.0) * c * x + alpha * alpha) * P[k] - 2.0 * (k + alpha) * k * (c + 2.0) * P[k - 1]) /
               (2.0 * (k + 1.0) * (k + alpha + 1.0) * c);
  }
}

template <class C>
void dubiner_eval(int p, C r, C s, std::vector<C>& out) {
  const C a = 2.0 * (1.0 + r) / (1.0 - s) - 1.0, b = s;
  std::vector<C> La, Lb;
  jacobi_all(p, 0.0, a, La);
  out.clear();
  for (int q = 0; q <= p; ++q)
    for (int i = q; i >= 0; --i) {
      const int j = q - i;
      jacobi_all(j, 2.0 * i + 1.0, b, Lb);
      C pw(1.0);
      for (int t = 0; t < i; ++t) pw = pw * (1.0 - b);
      const double na = 2.0 / (2.0 * i + 1.0), nb = pow(2.0, 2.0 * i + 2.0) / (2.0 * j + 2.0 * i + 2.0);
      out.push_back(sqrt(2.0) * (La[i] / sqrt(na)) * (Lb[j] / sqrt(nb)) * pw);
    }
}

// values and reference derivatives of every mode at (r, s)
void dubiner_point(int p, double r, double s, std::vector<double>& v, std::vector<double>& dr,
                   std::vector<double>& ds) {
  const double h = 1e-30;
  std::vector<std::complex<double>> a, b, c;
  dubiner_eval(p, std::complex<double>(r, 0.0), std::complex<double>(s, 0.0), a);
  dubiner_eval(p, std::complex<double>(r, h), std::complex<double>(s, 0.0), b);
  dubiner_eval(p, std::complex<double>(r, 0.0), std::complex<double>(s, h), c);
  v.resize(a.size());
  dr.resize(a.size());
  ds.resize(a.size());
  for (size_t i = 0; i < a.size(); ++i) {
    v[i] = a[i].real();
    dr[i] = b[i].imag() / h;
    ds[i] = c[i].imag() / h;
  }
}

// Gauss-Legendre by Newton on P_n (same construction as the structured mesh)
void gl_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    const double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  if (n == 1) {
    x[0] = 0.0;
    w[0] = 2.0;
  }
}

const double REF_V[3][2] = {{-1.0, -1.0}, {1.0, -1.0}, {-1.0, 1.0}};
const int REF_E[3][2] = {{0, 1}, {1, 2}, {2, 0}};

template <class T>
cudaError_t upload_vec(Mesh& M, const std::vector<double>& h, T** d) {
  std::vector<T> c(h.begin(), h.end());
  cudaError_t e = cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(c.size(), 1));
  if (e != cudaSuccess) return e;
  M.allocs.push_back(*d);
  return cudaMemcpy(*d, c.data(), sizeof(T) * c.size(), cudaMemcpyHostToDevice);
}

// ---------------------------------------------------------------- device
template <class T>
struct TriView {
  int E, nm, nb, nq, nqf;
  const int* nbr;   // [E][3] neighbour across local edge f
  const int* nbrf;  // [E][3] the neighbour's local edge
  const T* geo;     // [E][5]: Jinv[0][0], Jinv[0][1], Jinv[1][0], Jinv[1][1] (d xi_l / d x_k), |J|
  const T* egeo;    // [E][3][3]: outward normal n0, n1, |J_F| = edge length / 2
  const T* vphi;    // [nq][nm]
  const T* vdphi;   // [2][nq][nm] reference derivatives
  const T* vw;      // [nq] reference weights
  const T* ephi;    // [3][nqf][nm]
  const T* edphi;   // [3][2][nqf][nm]
  const T* ew;      // [nqf]
  const T* P;       // [3][nqf][nqf]
};

template <class S, class T, bool JVP>
__device__ __forceinline__ void tri_trace(const T* __restrict__ W, const T* __restrict__ V, size_t base, int nm,
                                          const T* phi, const T* d0, const T* d1, const T* Ji, S* u, S (*g)[2]) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    T a = T(0), b0 = T(0), b1 = T(0), ta = T(0), tb0 = T(0), tb1 = T(0);
    const T* w = W + base + (size_t)v * nm;
    const T* x = JVP ? V + base + (size_t)v * nm : nullptr;
    for (int i = 0; i < nm; ++i) {
      const T wi = w[i];
      a += wi * phi[i];
      b0 += wi * d0[i];
      b1 += wi * d1[i];
      if (JVP) {
        const T xi = x[i];
        ta += xi * phi[i];
        tb0 += xi * d0[i];
        tb1 += xi * d1[i];
      }
    }
    if constexpr (JVP) {
      u[v] = S(a, ta);
      g[v][0] = S(Ji[0] * b0 + Ji[2] * b1, Ji[0] * tb0 + Ji[2] * tb1);
      g[v][1] = S(Ji[1] * b0 + Ji[3] * b1, Ji[1] * tb0 + Ji[3] * tb1);
    } else {
      u[v] = a;
      g[v][0] = Ji[0] * b0 + Ji[2] * b1;
      g[v][1] = Ji[1] * b0 + Ji[3] * b1;
    }
  }
}

template <class S>
__device__ __forceinline__ auto part(const S& x) {
  if constexpr (std::is_arithmetic<S>::value)
    return x;
  else
    return x.d;   // the tangent of a dual number
}

// Roe flux with normal n: the e_0 flux in the frame (n, t), t = (-n1, n0)
template <class S, class T>
__device__ __forceinline__ void roe_normal(const S* uL, const S* uR, T n0, T n1, S* F, const Phys<T>& ph) {
  S a[4], b[4], Fr[4];
  a[0] = uL[0];
  a[1] = uL[1] * n0 + uL[2] * n1;
  a[2] = uL[2] * n0 - uL[1] * n1;
  a[3] = uL[3];
  b[0] = uR[0];
  b[1] = uR[1] * n0 + uR[2] * n1;
  b[2] = uR[2] * n0 - uR[1] * n1;
  b[3] = uR[3];
  roe_flux<2, 0, S, T>(a, b, Fr, ph);
  F[0] = Fr[0];
  F[1] = Fr[1] * n0 - Fr[2] * n1;
  F[2] = Fr[1] * n1 + Fr[2] * n0;
  F[3] = Fr[3];
}

// K(u) (a (x) n) = n0 K(u)(a (x) e0) + n1 K(u)(a (x) e1)
template <class S, class T>
__device__ __forceinline__ void visc_K_normal(const S* u, const S* a, T n0, T n1, S (*G)[2], const Phys<T>& ph) {
  S G0[4][2], G1[4][2];
  visc_K_rank1<2, 0, S, T>(u, a, G0, ph);
  visc_K_rank1<2, 1, S, T>(u, a, G1, ph);
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int k = 0; k < 2; ++k) G[v][k] = G0[v][k] * n0 + G1[v][k] * n1;
}

constexpr int TF_NS = 24;   // per face point: fp[4], GPn[4], GMn[4], Dr[4][2], fhat[4]

template <class T, bool JVP>
__global__ void __launch_bounds__(128) tri_face_kernel(TriView<T> tv, Phys<T> ph, const T* __restrict__ W,
                                                       const T* __restrict__ V, T* __restrict__ slots, int* status,
                                                       int fpc) {
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sb = reinterpret_cast<T*>(smem_raw);   // [fpc][nqf][TF_NS]
  const int nqf = tv.nqf, nm = tv.nm, nb = tv.nb;
  const long F = 3L * tv.E;
  for (long f0 = (long)blockIdx.x * fpc; f0 < F; f0 += (long)gridDim.x * fpc) {
    for (int t = threadIdx.x; t < fpc * nqf; t += blockDim.x) {
      const int lf = t / nqf, q = t - lf * nqf;
      const long gf = f0 + lf;
      if (gf >= F) continue;
      const int e = (int)(gf / 3), f = (int)(gf - 3L * e);
      const int en = tv.nbr[gf], fn = tv.nbrf[gf];
      const T* eg = tv.egeo + gf * 3;
      const T n0 = eg[0], n1 = eg[1];
      const T* JiP = tv.geo + (size_t)e * 5;
      const T* JiM = tv.geo + (size_t)en * 5;
      const int qm = nqf - 1 - q;
      S uP[4], gP[4][2], uM[4], gM[4][2];
      tri_trace<S, T, JVP>(W, V, (size_t)e * nb, nm, tv.ephi + ((size_t)f * nqf + q) * nm,
                           tv.edphi + (((size_t)f * 2 + 0) * nqf + q) * nm,
                           tv.edphi + (((size_t)f * 2 + 1) * nqf + q) * nm, JiP, uP, gP);
      tri_trace<S, T, JVP>(W, V, (size_t)en * nb, nm, tv.ephi + ((size_t)fn * nqf + qm) * nm,
                           tv.edphi + (((size_t)fn * 2 + 0) * nqf + qm) * nm,
                           tv.edphi + (((size_t)fn * 2 + 1) * nqf + qm) * nm, JiM, uM, gM);
      if (!physical<2>(uP, ph.gm1) || !physical<2>(uM, ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
      S Fr[4], cP0[4], cP1[4], cM0[4], cM1[4], jump[4], K[4][2];
      roe_normal<S, T>(uP, uM, n0, n1, Fr, ph);
      flux_visc_col<2, 0, S, T>(uP, gP, cP0, ph);
      flux_visc_col<2, 1, S, T>(uP, gP, cP1, ph);
      flux_visc_col<2, 0, S, T>(uM, gM, cM0, ph);
      flux_visc_col<2, 1, S, T>(uM, gM, cM1, ph);
      T* o = sb + (size_t)t * TF_NS;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        jump[v] = uP[v] - uM[v];
        o[v] = part(Fr[v] + T(0.5) * ((cP0[v] + cM0[v]) * n0 + (cP1[v] + cM1[v]) * n1));
      }
      visc_K_normal<S, T>(uP, jump, n0, n1, K, ph);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        o[4 + v] = part(K[v][0] * n0 + K[v][1] * n1);
        // dual term integrand 1/2 K(u+)(jump (x) n), contravariant: sum_k Jinv[l][k] D_k
        const S d0 = T(0.5) * K[v][0], d1 = T(0.5) * K[v][1];
        o[12 + 2 * v + 0] = part(d0 * JiP[0] + d1 * JiP[1]);
        o[12 + 2 * v + 1] = part(d0 * JiP[2] + d1 * JiP[3]);
      }
      visc_K_normal<S, T>(uM, jump, n0, n1, K, ph);
#pragma unroll
      for (int v = 0; v < 4; ++v) o[8 + v] = part(K[v][0] * n0 + K[v][1] * n1);
    }
    __syncthreads();
    // fhat = fp + eta {delta}.n at every point (liftings through P of each side)
    for (int t = threadIdx.x; t < fpc * nqf; t += blockDim.x) {
      const int lf = t / nqf, q2 = t - lf * nqf;
      const long gf = f0 + lf;
      if (gf >= F) continue;
      const int e = (int)(gf / 3), f = (int)(gf - 3L * e);
      const int en = tv.nbr[gf], fn = tv.nbrf[gf];
      const T JF = tv.egeo[gf * 3 + 2];
      const T clP = JF / (T(2) * tv.geo[(size_t)e * 5 + 4]), clM = JF / (T(2) * tv.geo[(size_t)en * 5 + 4]);
      const T* PP = tv.P + (size_t)f * nqf * nqf;
      const T* PM = tv.P + (size_t)fn * nqf * nqf;
      const T* base = sb + (size_t)lf * nqf * TF_NS;
      T sP[4] = {T(0), T(0), T(0), T(0)}, sM[4] = {T(0), T(0), T(0), T(0)};
      for (int q = 0; q < nqf; ++q) {
        const T wP = tv.ew[q] * PP[q * nqf + q2];
        const T wM = tv.ew[q] * PM[(nqf - 1 - q) * nqf + (nqf - 1 - q2)];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          sP[v] += wP * base[q * TF_NS + 4 + v];
          sM[v] += wM * base[q * TF_NS + 8 + v];
        }
      }
      T* o = sb + (size_t)t * TF_NS;
#pragma unroll
      for (int v = 0; v < 4; ++v) o[20 + v] = o[v] + ph.eta * T(0.5) * (clP * sP[v] + clM * sM[v]);
    }
    __syncthreads();
    // projection on the test functions of this triangle
    for (int t = threadIdx.x; t < fpc * nb; t += blockDim.x) {
      const int lf = t / nb, j = t - lf * nb, v = j / nm, i = j - v * nm;
      const long gf = f0 + lf;
      if (gf >= F) continue;
      const int f = (int)(gf % 3);
      const T* base = sb + (size_t)lf * nqf * TF_NS;
      T acc = T(0);
      for (int q = 0; q < nqf; ++q) {
        const T* o = base + q * TF_NS;
        acc += tv.ew[q] * (o[20 + v] * tv.ephi[((size_t)f * nqf + q) * nm + i] -
                           o[12 + 2 * v] * tv.edphi[(((size_t)f * 2 + 0) * nqf + q) * nm + i] -
                           o[12 + 2 * v + 1] * tv.edphi[(((size_t)f * 2 + 1) * nqf + q) * nm + i]);
      }
      slots[gf * nb + j] = tv.egeo[gf * 3 + 2] * acc;
    }
    __syncthreads();
  }
}

template <class T, bool JVP>
__global__ void __launch_bounds__(128) tri_volume_kernel(TriView<T> tv, Phys<T> ph, const T* __restrict__ W,
                                                         const T* __restrict__ V, const T* __restrict__ slots,
                                                         const T* __restrict__ Src, T sigma, T* __restrict__ out,
                                                         int* status, int epc) {
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Fs = reinterpret_cast<T*>(smem_raw);   // [epc][2][4][nq]: |J| w_q sum_k Jinv[l][k] F[v][k]
  const int nq = tv.nq, nm = tv.nm, nb = tv.nb, E = tv.E;
  for (long e0 = (long)blockIdx.x * epc; e0 < E; e0 += (long)gridDim.x * epc) {
    for (int t = threadIdx.x; t < epc * nq; t += blockDim.x) {
      const int le = t / nq, q = t - le * nq;
      const long e = e0 + le;
      if (e >= E) continue;
      const T* Ji = tv.geo + (size_t)e * 5;
      S u[4], g[4][2], Fl[4][2];
      tri_trace<S, T, JVP>(W, V, (size_t)e * nb, nm, tv.vphi + (size_t)q * nm, tv.vdphi + (size_t)q * nm,
                           tv.vdphi + ((size_t)nq + q) * nm, Ji, u, g);
      if (!physical<2>(u, ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
      flux_total<2, S, T>(u, g, Fl, ph);
      const T wd = tv.vw[q] * Ji[4];
      T* o = Fs + (size_t)le * 8 * nq;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        o[(0 * 4 + v) * nq + q] = wd * part(Fl[v][0] * Ji[0] + Fl[v][1] * Ji[1]);
        o[(1 * 4 + v) * nq + q] = wd * part(Fl[v][0] * Ji[2] + Fl[v][1] * Ji[3]);
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < epc * nb; t += blockDim.x) {
      const int le = t / nb, j = t - le * nb, v = j / nm, i = j - v * nm;
      const long e = e0 + le;
      if (e >= E) continue;
      const T* o = Fs + (size_t)le * 8 * nq;
      T acc = T(0);
      for (int q = 0; q < nq; ++q)
        acc -= o[(0 * 4 + v) * nq + q] * tv.vdphi[(size_t)q * nm + i] +
               o[(1 * 4 + v) * nq + q] * tv.vdphi[((size_t)nq + q) * nm + i];
      acc += slots[(e * 3 + 0) * nb + j];
      acc += slots[(e * 3 + 1) * nb + j];
      acc += slots[(e * 3 + 2) * nb + j];
      if (JVP)
        acc += sigma * tv.geo[(size_t)e * 5 + 4] * V[e * nb + j];
      else if (Src)
        acc -= Src[e * nb + j];
      out[e * nb + j] = acc;
    }
    __syncthreads();
  }
}

template <class T>
const TriTab<T>& tri_tab(const Mesh& M) {
  if constexpr (std::is_same<T, double>::value)
    return M.tr64;
  else
    return M.tr32;
}

template <class T>
TriView<T> tri_view(const Mesh& M) {
  const TriTab<T>& tb = tri_tab<T>(M);
  TriView<T> v;
  v.E = M.E;
  v.nm = M.nm;
  v.nb = M.nb;
  v.nq = M.nq;
  v.nqf = M.nqf;
  v.nbr = M.tnbr;
  v.nbrf = M.tnbrf;
  v.geo = tb.geo;
  v.egeo = tb.egeo;
  v.vphi = tb.vphi;
  v.vdphi = tb.vdphi;
  v.vw = tb.vw;
  v.ephi = tb.ephi;
  v.edphi = tb.edphi;
  v.ew = tb.ew;
  v.P = tb.P;
  return v;
}

}  // namespace

template <class T>
cudaError_t launch_residual_tri(const Mesh& M, const T* W, const T* V, const T* S, T sigma, bool jvp, T* out,
                                cudaStream_t st) {
  const TriView<T> tv = tri_view<T>(M);
  const Phys<T> ph = M.phys_t<T>();
  T* slots = std::is_same<T, double>::value ? (T*)M.t64.slots : (T*)M.t32.slots;
  const int fpc = std::max(1, 128 / M.nqf);
  const long F = 3L * M.E;
  const int gf = (int)std::min<long>((F + fpc - 1) / fpc, 1L << 20);
  const size_t fsm = (size_t)fpc * M.nqf * TF_NS * sizeof(T);
  note_launch();
  if (jvp)
    tri_face_kernel<T, true><<<gf, 128, fsm, st>>>(tv, ph, W, V, slots, M.status, fpc);
  else
    tri_face_kernel<T, false><<<gf, 128, fsm, st>>>(tv, ph, W, nullptr, slots, M.status, fpc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int epc = std::max(1, 128 / M.nq);
  const int gv = (int)std::min<long>((M.E + epc - 1) / epc, 1L << 20);
  const size_t vsm = (size_t)epc * 8 * M.nq * sizeof(T);
  note_launch();
  if (jvp)
    tri_volume_kernel<T, true><<<gv, 128, vsm, st>>>(tv, ph, W, V, slots, nullptr, sigma, out, M.status, epc);
  else
    tri_volume_kernel<T, false><<<gv, 128, vsm, st>>>(tv, ph, W, nullptr, slots, S, sigma, out, M.status, epc);
  return cudaGetLastError();
}
template cudaError_t launch_residual_tri<double>(const Mesh&, const double*, const double*, const double*, double,
                                                 bool, double*, cudaStream_t);
template cudaError_t launch_residual_tri<float>(const Mesh&, const float*, const float*, const float*, float, bool,
                                                float*, cudaStream_t);

// ---------------------------------------------------------------- blocks
// Block probing by coloured JVPs (Sec. 5.1 blocks of the iteration matrix):
// the seed is the unit direction jj on every triangle of colour c.  No two
// triangles of one colour are neighbours, so the JVP's rows on colour c are
// column jj of D_e = dR_e/dW_e + sigma |J_e| I, and the face slot of edge f of
// a triangle whose neighbour across f has colour c is column jj of the
// neighbour block (that slot depends on the two triangles only).
namespace {

template <class T>
__global__ void tri_seed_kernel(long N, int nb, const int* __restrict__ colour, int c, int jj, T* __restrict__ seed) {
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
    const long e = n / nb;
    seed[n] = (colour[e] == c && n - e * nb == jj) ? T(1) : T(0);
  }
}

template <class T>
__global__ void tri_gather_kernel(int E, int nb, int nm, const int* __restrict__ colour, const int* __restrict__ nbr,
                                  int c, int jj, const T* __restrict__ out, const T* __restrict__ slots, T* D,
                                  size_t dstride, T* O, int nmc) {
  const int nbc = 4 * nmc;
  const long nD = (long)E * nb, nO = O ? (long)E * 3 * nbc : 0;
  const int jv = jj / nm, ji = jj - jv * nm;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nD + nO; t += (long)gridDim.x * blockDim.x) {
    if (t < nD) {
      const long e = t / nb;
      const int r = (int)(t - e * nb);
      if (colour[e] == c) D[e * dstride + (size_t)r * nb + jj] = out[t];
    } else {
      const long t2 = t - nD, ef = t2 / nbc;   // ef = 3 e + f
      const int rc = (int)(t2 - ef * nbc);
      const long e = ef / 3;
      const int k = nbr[ef];
      if (ji < nmc && k != e && colour[k] == c) {
        const int rv = rc / nmc, ri = rc - rv * nmc;
        O[ef * nbc * nbc + (size_t)rc * nbc + jv * nmc + ji] = slots[ef * nb + rv * nm + ri];
      }
    }
  }
}

}  // namespace

template <class T>
cudaError_t launch_probe_blocks_tri(const Mesh& M, const T* W, T sigma, T* D, size_t dstride, T* O, int nmc,
                                    T* seed, T* out, cudaStream_t st) {
  const long N = (long)M.E * M.nb;
  const T* slots = std::is_same<T, double>::value ? (const T*)M.t64.slots : (const T*)M.t32.slots;
  const int gs = (int)std::min<long>((N + 255) / 256, 4096);
  const long ng = N + (O ? (long)M.E * 3 * 4 * nmc : 0);
  const int gg = (int)std::min<long>((ng + 255) / 256, 4096);
  for (int c = 0; c < M.tncol; ++c)
    for (int jj = 0; jj < M.nb; ++jj) {
      note_launch();
      tri_seed_kernel<T><<<gs, 256, 0, st>>>(N, M.nb, M.tcolour, c, jj, seed);
      cudaError_t e = launch_residual_tri<T>(M, W, seed, nullptr, sigma, true, out, st);
      if (e != cudaSuccess) return e;
      note_launch();
      tri_gather_kernel<T><<<gg, 256, 0, st>>>(M.E, M.nb, M.nm, M.tcolour, M.tnbr, c, jj, out, slots, D, dstride, O,
                                               nmc);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  return cudaSuccess;
}
template cudaError_t launch_probe_blocks_tri<double>(const Mesh&, const double*, double, double*, size_t, double*, int,
                                                     double*, double*, cudaStream_t);
template cudaError_t launch_probe_blocks_tri<float>(const Mesh&, const float*, float, float*, size_t, float*, int,
                                                    float*, float*, cudaStream_t);

// ---------------------------------------------------------------- mesh build
namespace {

template <class T>
cudaError_t upload_tri_tables(Mesh& M, TriTab<T>& tb, const std::vector<double>* h) {
  cudaError_t e;
  if ((e = upload_vec<T>(M, h[0], &tb.geo)) != cudaSuccess || (e = upload_vec<T>(M, h[1], &tb.egeo)) != cudaSuccess ||
      (e = upload_vec<T>(M, h[2], &tb.vphi)) != cudaSuccess || (e = upload_vec<T>(M, h[3], &tb.vdphi)) != cudaSuccess ||
      (e = upload_vec<T>(M, h[4], &tb.vw)) != cudaSuccess || (e = upload_vec<T>(M, h[5], &tb.ephi)) != cudaSuccess ||
      (e = upload_vec<T>(M, h[6], &tb.edphi)) != cudaSuccess || (e = upload_vec<T>(M, h[7], &tb.ew)) != cudaSuccess ||
      (e = upload_vec<T>(M, h[8], &tb.P)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

template <class T>
cudaError_t alloc_scratch(Mesh& M, Tables<T>& t) {
  const size_t N = (size_t)M.E * M.nb;
  T** bufs[4] = {&t.slots, &t.fd_w, &t.fd_r, &t.fd_o};
  const size_t n[4] = {3 * N, N, N, N};
  for (int i = 0; i < 4; ++i) {
    cudaError_t e = cudaMalloc((void**)bufs[i], sizeof(T) * std::max<size_t>(n[i], 1));
    if (e != cudaSuccess) return e;
    M.allocs.push_back(*bufs[i]);
  }
  return cudaSuccess;
}

dg_status build_tri(Mesh& M, const dg_tri_desc* d, const dg_physics* ph) {
  memset(&M.desc, 0, sizeof(M.desc));
  M.desc.dim = 2;
  M.desc.p = d->p;
  M.desc.nq1d = d->nq1d;
  M.phys = *ph;
  if (!(M.phys.eta_br2 > 0.0)) M.phys.eta_br2 = 4.0;   // n_faces + 1 of a triangle
  M.kind = DG_MESH_TRI;
  M.d = 2;
  M.m = 4;
  M.p = d->p;
  M.nq1d = d->nq1d > 0 ? d->nq1d : d->p + 2;
  M.nm = (M.p + 1) * (M.p + 2) / 2;
  M.nb = M.m * M.nm;
  M.nq = M.nq1d * M.nq1d;
  M.nqf = M.nq1d;
  M.E = d->n_tri;
  M.detJ = 0.0;   // varies per triangle
  const int E = M.E, p = M.p, nq1 = M.nq1d, nm = M.nm;
  const double Lx = d->hi[0] - d->lo[0], Ly = d->hi[1] - d->lo[1];
  // geometry
  std::vector<double> geo((size_t)E * 5), egeo((size_t)E * 9);
  for (int e = 0; e < E; ++e) {
    double Vx[3], Vy[3];
    for (int k = 0; k < 3; ++k) {
      const int id = d->tri[3 * e + k];
      if (id < 0 || id >= d->n_vert) return DG_ERR_INVALID;
      Vx[k] = d->X[2 * id] + d->shift[(3 * e + k) * 2 + 0] * Lx;
      Vy[k] = d->X[2 * id + 1] + d->shift[(3 * e + k) * 2 + 1] * Ly;
    }
    const double J00 = (Vx[1] - Vx[0]) / 2, J01 = (Vx[2] - Vx[0]) / 2;
    const double J10 = (Vy[1] - Vy[0]) / 2, J11 = (Vy[2] - Vy[0]) / 2;
    const double det = J00 * J11 - J01 * J10;
    if (!(det > 0.0)) return DG_ERR_INVALID;   // clockwise or degenerate
    // Jinv[l][k] = d xi_l / d x_k
    geo[(size_t)e * 5 + 0] = J11 / det;
    geo[(size_t)e * 5 + 1] = -J01 / det;
    geo[(size_t)e * 5 + 2] = -J10 / det;
    geo[(size_t)e * 5 + 3] = J00 / det;
    geo[(size_t)e * 5 + 4] = det;
    for (int f = 0; f < 3; ++f) {
      const int a = REF_E[f][0], b = REF_E[f][1];
      const double dx = Vx[b] - Vx[a], dy = Vy[b] - Vy[a], L = sqrt(dx * dx + dy * dy);
      egeo[((size_t)e * 3 + f) * 3 + 0] = dy / L;
      egeo[((size_t)e * 3 + f) * 3 + 1] = -dx / L;
      egeo[((size_t)e * 3 + f) * 3 + 2] = L / 2.0;
    }
  }
  // connectivity: (vertex ids, relative lattice shift) of every edge
  using Key = std::tuple<int, int, int, int>;
  std::map<Key, std::vector<int>> edges;
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 3; ++f) {
      const int a = REF_E[f][0], b = REF_E[f][1];
      const int ga = d->tri[3 * e + a], gb = d->tri[3 * e + b];
      const int sx = d->shift[(3 * e + b) * 2 + 0] - d->shift[(3 * e + a) * 2 + 0];
      const int sy = d->shift[(3 * e + b) * 2 + 1] - d->shift[(3 * e + a) * 2 + 1];
      const Key k1(ga, gb, sx, sy), k2(gb, ga, -sx, -sy);
      edges[std::min(k1, k2)].push_back(3 * e + f);
    }
  std::vector<int> nbr((size_t)E * 3, -1), nbrf((size_t)E * 3, -1);
  for (auto& kv : edges) {
    if (kv.second.size() != 2) return DG_ERR_INVALID;
    const int a = kv.second[0], b = kv.second[1];
    nbr[a] = b / 3;
    nbrf[a] = b % 3;
    nbr[b] = a / 3;
    nbrf[b] = a % 3;
  }
  // tables
  std::vector<double> xg, wg;
  gl_rule(nq1, xg, wg);
  std::vector<double> vphi((size_t)M.nq * nm), vdphi((size_t)2 * M.nq * nm), vw(M.nq);
  std::vector<double> v, dr, ds;
  for (int ib = 0; ib < nq1; ++ib)
    for (int ia = 0; ia < nq1; ++ia) {
      const int q = ia + nq1 * ib;
      const double a = xg[ia], b = xg[ib];
      const double r = (1.0 + a) * (1.0 - b) / 2.0 - 1.0, s = b;
      vw[q] = wg[ia] * wg[ib] * (1.0 - b) / 2.0;
      dubiner_point(p, r, s, v, dr, ds);
      for (int i = 0; i < nm; ++i) {
        vphi[(size_t)q * nm + i] = v[i];
        vdphi[(size_t)q * nm + i] = dr[i];
        vdphi[((size_t)M.nq + q) * nm + i] = ds[i];
      }
    }
  const int nqf = M.nqf;
  std::vector<double> ephi((size_t)3 * nqf * nm), edphi((size_t)3 * 2 * nqf * nm), Pm((size_t)3 * nqf * nqf);
  for (int f = 0; f < 3; ++f) {
    const double* va = REF_V[REF_E[f][0]];
    const double* vb = REF_V[REF_E[f][1]];
    for (int q = 0; q < nqf; ++q) {
      const double t = xg[q];
      const double r = va[0] * (1.0 - t) / 2.0 + vb[0] * (1.0 + t) / 2.0;
      const double s = va[1] * (1.0 - t) / 2.0 + vb[1] * (1.0 + t) / 2.0;
      dubiner_point(p, r, s, v, dr, ds);
      for (int i = 0; i < nm; ++i) {
        ephi[((size_t)f * nqf + q) * nm + i] = v[i];
        edphi[(((size_t)f * 2 + 0) * nqf + q) * nm + i] = dr[i];
        edphi[(((size_t)f * 2 + 1) * nqf + q) * nm + i] = ds[i];
      }
    }
    for (int q = 0; q < nqf; ++q)
      for (int q2 = 0; q2 < nqf; ++q2) {
        double s = 0.0;
        for (int i = 0; i < nm; ++i) s += ephi[((size_t)f * nqf + q) * nm + i] * ephi[((size_t)f * nqf + q2) * nm + i];
        Pm[((size_t)f * nqf + q) * nqf + q2] = s;
      }
  }
  const std::vector<double> h[9] = {geo, egeo, vphi, vdphi, vw, ephi, edphi, wg, Pm};
  if (upload_tri_tables<double>(M, M.tr64, h) != cudaSuccess || upload_tri_tables<float>(M, M.tr32, h) != cudaSuccess)
    return DG_ERR_OOM;
  if (cudaMalloc((void**)&M.tnbr, sizeof(int) * E * 3) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.tnbr);
  if (cudaMalloc((void**)&M.tnbrf, sizeof(int) * E * 3) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.tnbrf);
  if (cudaMemcpy(M.tnbr, nbr.data(), sizeof(int) * E * 3, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(M.tnbrf, nbrf.data(), sizeof(int) * E * 3, cudaMemcpyHostToDevice) != cudaSuccess)
    return DG_ERR_CUDA;
  // greedy colouring in index order (no two face neighbours share a colour)
  std::vector<int> col(E, 0);
  M.tncol = 0;
  for (int e = 0; e < E; ++e) {
    int c = 0;
    for (bool clash = true; clash; ) {
      clash = false;
      for (int f = 0; f < 3; ++f) {
        const int k = nbr[(size_t)e * 3 + f];
        if (k < e && col[k] == c) clash = true;
      }
      if (clash) ++c;
    }
    col[e] = c;
    M.tncol = std::max(M.tncol, c + 1);
  }
  if (cudaMalloc((void**)&M.tcolour, sizeof(int) * E) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.tcolour);
  if (cudaMemcpy(M.tcolour, col.data(), sizeof(int) * E, cudaMemcpyHostToDevice) != cudaSuccess) return DG_ERR_CUDA;
  if (alloc_scratch<double>(M, M.t64) != cudaSuccess || alloc_scratch<float>(M, M.t32) != cudaSuccess)
    return DG_ERR_OOM;
  if (cudaMalloc((void**)&M.status, sizeof(int)) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.status);
  if (cudaMemset(M.status, 0, sizeof(int)) != cudaSuccess) return DG_ERR_CUDA;
  if (cudaMalloc((void**)&M.scal, 16 * sizeof(double)) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.scal);
  if (cudaMalloc((void**)&M.partials, 2 * 1024 * sizeof(double)) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.partials);
  return DG_OK;
}

}  // namespace

}  // namespace dgk

extern "C" dg_status dg_mesh_create_tri(const dg_tri_desc* desc, const dg_physics* phys, void* stream,
                                        dg_mesh* out) {
  (void)stream;
  if (!out) return DG_ERR_INVALID;
  *out = nullptr;
  if (!desc || !phys || !desc->X || !desc->tri || !desc->shift) return DG_ERR_INVALID;
  if (desc->n_vert < 3 || desc->n_tri < 2 || desc->n_tri > (1 << 24)) return DG_ERR_INVALID;
  if (desc->p < 0 || desc->p > 8) return DG_ERR_INVALID;
  const int nq1 = desc->nq1d > 0 ? desc->nq1d : desc->p + 2;
  if (nq1 < desc->p + 1 || nq1 > 12) return DG_ERR_INVALID;
  if (!(desc->hi[0] > desc->lo[0]) || !(desc->hi[1] > desc->lo[1])) return DG_ERR_INVALID;
  if (!(phys->gamma > 1.0) || !(phys->Rgas > 0.0) || phys->mu < 0.0 || !(phys->Pr > 0.0) ||
      phys->roe_delta < 0.0 || phys->eta_br2 < 0.0)
    return DG_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  dg_mesh h = new dg_mesh_s();
  dg_status s = dgk::build_tri(h->m, desc, phys);
  if (s != DG_OK) {
    dgk::free_mesh(h->m);
    delete h;
    return s;
  }
  *out = h;
  return DG_OK;
}
