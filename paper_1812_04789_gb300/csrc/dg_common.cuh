// Shared device definitions: forward-mode dual numbers, pointwise compressible
// Navier-Stokes physics (Sec. 2 closure, Sec. 3.1 fluxes), device mesh view.
//
// Every pointwise routine is templated on the scalar S (T = float/double for a
// residual, Dual<T> for a Jacobian-vector product: value + directional
// derivative, so the JVP is the exact linearisation of the discrete residual)
// and on the dimension D (2 or 3); m = D + 2 conservative variables
// (rho, rho v_1..rho v_D, rho e0).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgk {

// 8 consecutive BF16 values (16 bytes, read-only, not kept in L1) widened to
// FP32: a BF16 value is the upper half of the FP32 with the same bits.
__device__ __forceinline__ void ld_bf16x8(const unsigned short* p, float* v) {
  unsigned a, b, c, d;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
               : "l"(p));
  v[0] = __uint_as_float(a << 16);
  v[1] = __uint_as_float(a & 0xffff0000u);
  v[2] = __uint_as_float(b << 16);
  v[3] = __uint_as_float(b & 0xffff0000u);
  v[4] = __uint_as_float(c << 16);
  v[5] = __uint_as_float(c & 0xffff0000u);
  v[6] = __uint_as_float(d << 16);
  v[7] = __uint_as_float(d & 0xffff0000u);
}

// ----------------------------------------------------------------- duals
template <class T>
struct Dual {
  T v, d;
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(T a) : v(a), d(T(0)) {}
  __host__ __device__ Dual(T a, T b) : v(a), d(b) {}
};
template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
// one division per quotient: the tangent reuses the reciprocal of the value
template <class T> __host__ __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  const T r = T(1) / b.v;
  const T q = a.v * r;
  return Dual<T>(q, (a.d - q * b.d) * r);
}
template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return Dual<T>(a.v + b, a.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return Dual<T>(a + b.v, b.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return Dual<T>(a.v - b, a.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return Dual<T>(a - b.v, -b.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return Dual<T>(a.v * b, a.d * b); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return Dual<T>(a * b.v, a * b.d); }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator/(Dual<T> a, T b) {
  const T r = T(1) / b;
  return Dual<T>(a.v * r, a.d * r);
}
template <class T> __host__ __device__ __forceinline__ Dual<T> operator/(T a, Dual<T> b) {
  const T r = T(1) / b.v;
  const T q = a * r;
  return Dual<T>(q, -q * b.d * r);
}
template <class T> __host__ __device__ __forceinline__ Dual<T> dsqrt(Dual<T> a) {
  const T s = sqrt(a.v);
  return Dual<T>(s, a.d * (T(0.5) / s));
}
__host__ __device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__host__ __device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }

template <class T> __host__ __device__ __forceinline__ T val(Dual<T> a) { return a.v; }
__host__ __device__ __forceinline__ double val(double a) { return a; }
__host__ __device__ __forceinline__ float val(float a) { return a; }
template <class T> __host__ __device__ __forceinline__ T tan_part(Dual<T> a) { return a.d; }
__host__ __device__ __forceinline__ double tan_part(double a) { return a; }
__host__ __device__ __forceinline__ float tan_part(float a) { return a; }

// |x| continued so that the derivative at x = 0 is +1 (x >= 0 is "positive")
template <class S> __host__ __device__ __forceinline__ S sabs(S x) { return val(x) >= 0 ? x : -x; }

// ----------------------------------------------------------------- physics
template <class T>
struct Phys {
  T gamma, gm1, Pr, mu, Rgas, eta, roe_delta, kappa;  // kappa = mu c_p / Pr
};

// Inviscid flux column k: (rho v_k, rho v_j v_k + p delta_jk, rho v_k h0)
// Full tensor F_c + F_v at a point: F[v][k].
template <int D, class S, class T>
__host__ __device__ __forceinline__ void flux_total(const S* u, const S (*g)[D], S (*F)[D],
                                           const Phys<T>& ph) {
  constexpr int M = D + 2;
  S rho = u[0];
  S ir = T(1) / rho;
  S vel[D];
#pragma unroll
  for (int j = 0; j < D; ++j) vel[j] = u[1 + j] * ir;
  S e0 = u[M - 1] * ir;
  S q2 = vel[0] * vel[0];
#pragma unroll
  for (int j = 1; j < D; ++j) q2 = q2 + vel[j] * vel[j];
  S p = ph.gm1 * (u[M - 1] - T(0.5) * rho * q2);
  S h0 = e0 + p * ir;
  // primitive gradients from conservative ones
  S gv[D][D], gT[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int j = 0; j < D; ++j) gv[j][k] = (g[1 + j][k] - vel[j] * g[0][k]) * ir;
    S ge = (g[M - 1][k] - e0 * g[0][k]) * ir;
    S s = vel[0] * gv[0][k];
#pragma unroll
    for (int j = 1; j < D; ++j) s = s + vel[j] * gv[j][k];
    gT[k] = (ph.gm1 / ph.Rgas) * (ge - s);
  }
  S div = gv[0][0];
#pragma unroll
  for (int j = 1; j < D; ++j) div = div + gv[j][j];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    F[0][k] = u[1 + k];
    S tv = T(0);                               // sum_j v_j tau_jk
#pragma unroll
    for (int j = 0; j < D; ++j) {
      S tau = ph.mu * (gv[j][k] + gv[k][j]);
      if (j == k) tau = tau - (T(2) / T(3)) * ph.mu * div;
      S inv = u[1 + j] * vel[k];
      if (j == k) inv = inv + p;
      F[1 + j][k] = inv - tau;
      tv = tv + vel[j] * tau;
    }
    F[M - 1][k] = rho * vel[k] * h0 - (tv + ph.kappa * gT[k]);
  }
}

// Viscous flux only (F_v = -(0, tau, v.tau - q)), column k, for face averages.
template <int D, int k, class S, class T>
__host__ __device__ __forceinline__ void flux_visc_col(const S* u, const S (*g)[D], S* Fk,
                                              const Phys<T>& ph) {
  constexpr int M = D + 2;
  S ir = T(1) / u[0];
  S vel[D];
#pragma unroll
  for (int j = 0; j < D; ++j) vel[j] = u[1 + j] * ir;
  S e0 = u[M - 1] * ir;
  S gv[D][D];
  S gTk = T(0);
#pragma unroll
  for (int kk = 0; kk < D; ++kk) {
#pragma unroll
    for (int j = 0; j < D; ++j) gv[j][kk] = (g[1 + j][kk] - vel[j] * g[0][kk]) * ir;
  }
  {
    S ge = (g[M - 1][k] - e0 * g[0][k]) * ir;
    S s = vel[0] * gv[0][k];
#pragma unroll
    for (int j = 1; j < D; ++j) s = s + vel[j] * gv[j][k];
    gTk = (ph.gm1 / ph.Rgas) * (ge - s);
  }
  S div = gv[0][0];
#pragma unroll
  for (int j = 1; j < D; ++j) div = div + gv[j][j];
  Fk[0] = T(0);
  S tv = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    S tau = ph.mu * (gv[j][k] + gv[k][j]);
    if (j == k) tau = tau - (T(2) / T(3)) * ph.mu * div;
    Fk[1 + j] = -tau;
    tv = tv + vel[j] * tau;
  }
  Fk[M - 1] = -(tv + ph.kappa * gTk);
}

// G = K(u) (a (x) e_k) = -F_v(u, a (x) e_k): the viscous operator applied to the
// rank-one gradient a e_k^T (full tensor G[v][kk]).  Used by the BR2 lifting
// (eq. re) and the dual-consistency term of eq. dg_ns.
template <int D, int k, class S, class T>
__host__ __device__ __forceinline__ void visc_K_rank1(const S* u, const S* a, S (*G)[D],
                                             const Phys<T>& ph) {
  constexpr int M = D + 2;
  S ir = T(1) / u[0];
  S vel[D], av[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vel[j] = u[1 + j] * ir;
    av[j] = (a[1 + j] - vel[j] * a[0]) * ir;     // d v_j along e_k
  }
  S e0 = u[M - 1] * ir;
  S ae = (a[M - 1] - e0 * a[0]) * ir;
  S s = vel[0] * av[0];
#pragma unroll
  for (int j = 1; j < D; ++j) s = s + vel[j] * av[j];
  S aT = (ph.gm1 / ph.Rgas) * (ae - s);
  S div = av[k];
#pragma unroll
  for (int kk = 0; kk < D; ++kk) {
    G[0][kk] = T(0);
    S tv = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      S tau = T(0);
      if (kk == k) tau = tau + ph.mu * av[j];
      if (j == k) tau = tau + ph.mu * av[kk];
      if (j == kk) tau = tau - (T(2) / T(3)) * ph.mu * div;
      G[1 + j][kk] = tau;
      tv = tv + vel[j] * tau;
    }
    G[M - 1][kk] = tv + ((kk == k) ? ph.kappa * aT : S(T(0)));
  }
}

template <class S, class T>
__host__ __device__ __forceinline__ S entropy_fixed_abs(S lam, S delta) {
  S a = sabs(lam);
  if (val(delta) > T(0) && val(a) < val(delta)) return (lam * lam + delta * delta) / (T(2) * delta);
  return a;
}

// Roe flux with normal +e_k: 1/2 (F_c(uL) + F_c(uR)).e_k - 1/2 |A_Roe| (uR - uL).
template <int D, int k, class S, class T>
__host__ __device__ __forceinline__ void roe_flux(const S* uL, const S* uR, S* Fh,
                                         const Phys<T>& ph) {
  constexpr int M = D + 2;
  S rL = uL[0], rR = uR[0];
  S irL = T(1) / rL, irR = T(1) / rR;
  S vL[D], vR[D];
  S q2L = T(0), q2R = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vL[j] = uL[1 + j] * irL;
    vR[j] = uR[1 + j] * irR;
    q2L = q2L + vL[j] * vL[j];
    q2R = q2R + vR[j] * vR[j];
  }
  S pL = ph.gm1 * (uL[M - 1] - T(0.5) * rL * q2L);
  S pR = ph.gm1 * (uR[M - 1] - T(0.5) * rR * q2R);
  S hL = (uL[M - 1] + pL) * irL;
  S hR = (uR[M - 1] + pR) * irR;
  S sL = dsqrt(rL), sR = dsqrt(rR);
  S isum = T(1) / (sL + sR);
  S rho = sL * sR;
  S vel[D];
  S q2 = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vel[j] = (sL * vL[j] + sR * vR[j]) * isum;
    q2 = q2 + vel[j] * vel[j];
  }
  S h0 = (sL * hL + sR * hR) * isum;
  S c2 = ph.gm1 * (h0 - T(0.5) * q2);
  S c = dsqrt(c2);
  S vn = vel[k];
  S dr = rR - rL, dp = pR - pL;
  S dv[D];
  S vdv = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    dv[j] = vR[j] - vL[j];
    vdv = vdv + vel[j] * dv[j];
  }
  S dvn = dv[k];
  S ic2 = T(1) / c2;
  S a1 = (dp - rho * c * dvn) * (T(0.5) * ic2);
  S a3 = (dp + rho * c * dvn) * (T(0.5) * ic2);
  S a2 = dr - dp * ic2;
  S delta = ph.roe_delta * c;
  S l1 = entropy_fixed_abs<S, T>(vn - c, delta) * a1;
  S l2 = entropy_fixed_abs<S, T>(vn, delta);
  S l3 = entropy_fixed_abs<S, T>(vn + c, delta) * a3;
  // inviscid flux column k of both states
  Fh[0] = T(0.5) * (uL[1 + k] + uR[1 + k]) - T(0.5) * (l1 + l3 + l2 * a2);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    S fl = uL[1 + j] * vL[k];
    S fr = uR[1 + j] * vR[k];
    if (j == k) {
      fl = fl + pL;
      fr = fr + pR;
    }
    S dis = l1 * vel[j] + l3 * vel[j] + l2 * (a2 * vel[j] + rho * dv[j]);
    if (j == k) dis = dis - l1 * c + l3 * c - l2 * rho * dvn;
    Fh[1 + j] = T(0.5) * (fl + fr) - T(0.5) * dis;
  }
  S disE = l1 * (h0 - c * vn) + l3 * (h0 + c * vn) + l2 * (a2 * T(0.5) * q2 + rho * (vdv - vn * dvn));
  Fh[M - 1] = T(0.5) * (rL * vL[k] * hL + rR * vR[k] * hR) - T(0.5) * disE;
}

// Pointwise physics of one face point, normal +e_k from L (its xi_k = +1 side)
// to R.  fp = Roe(uL, uR) + {F_v}.e_k; with jump = uL - uR,
// GLn/GRn = normal column of K(uL)/K(uR) (jump (x) e_k) (the BR2 lifting
// integrand of eq. re) and DL/DR = half the full tensors (the dual-consistency
// term of eq. dg_ns, (u+ - uhat) = jump/2).  The direction is a compile-time
// constant: no local array is indexed at run time.
template <int D, int k, class S, class T>
__host__ __device__ __forceinline__ void face_point(const S* uL, const S (*gL)[D], const S* uR,
                                                    const S (*gR)[D], const Phys<T>& ph, S* fp, S* GLn,
                                                    S* GRn, S (*DL)[D], S (*DR)[D]) {
  constexpr int M = D + 2;
  S jump[M], Fr[M], FvL[M], FvR[M], G[M][D];
#pragma unroll
  for (int v = 0; v < M; ++v) jump[v] = uL[v] - uR[v];
  roe_flux<D, k, S, T>(uL, uR, Fr, ph);
  flux_visc_col<D, k, S, T>(uL, gL, FvL, ph);
  flux_visc_col<D, k, S, T>(uR, gR, FvR, ph);
#pragma unroll
  for (int v = 0; v < M; ++v) fp[v] = Fr[v] + T(0.5) * (FvL[v] + FvR[v]);
  visc_K_rank1<D, k, S, T>(uL, jump, G, ph);
#pragma unroll
  for (int v = 0; v < M; ++v) {
    GLn[v] = G[v][k];
#pragma unroll
    for (int kk = 0; kk < D; ++kk) DL[v][kk] = T(0.5) * G[v][kk];
  }
  visc_K_rank1<D, k, S, T>(uR, jump, G, ph);
#pragma unroll
  for (int v = 0; v < M; ++v) {
    GRn[v] = G[v][k];
#pragma unroll
    for (int kk = 0; kk < D; ++kk) DR[v][kk] = T(0.5) * G[v][kk];
  }
}

template <int D, class S, class T>
__host__ __device__ __forceinline__ void face_point_k(int k, const S* uL, const S (*gL)[D], const S* uR,
                                                      const S (*gR)[D], const Phys<T>& ph, S* fp, S* GLn,
                                                      S* GRn, S (*DL)[D], S (*DR)[D]) {
  if (k == 0) {
    face_point<D, 0, S, T>(uL, gL, uR, gR, ph, fp, GLn, GRn, DL, DR);
  } else if (k == 1) {
    face_point<D, 1, S, T>(uL, gL, uR, gR, ph, fp, GLn, GRn, DL, DR);
  } else {
    if constexpr (D == 3) face_point<D, 2, S, T>(uL, gL, uR, gR, ph, fp, GLn, GRn, DL, DR);
  }
}

// rho > 0 and p > 0 of a point state (primal values)
template <int D, class S, class T>
__host__ __device__ __forceinline__ bool physical(const S* u, T gm1) {
  constexpr int M = D + 2;
  T r = val(u[0]);
  T q = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) q += val(u[1 + j]) * val(u[1 + j]);
  T p = gm1 * (val(u[M - 1]) - T(0.5) * q / r);
  return r > T(0) && p > T(0);
}

// ----------------------------------------------------------------- mesh view
template <class T>
struct MeshView {
  int d, m, nm, nb, nq, nqf, E;
  int n[3];
  const int* nbr;          // [E][d][2]   face neighbours (side 0: -e_k, side 1: +e_k)
  const T* vphiT;          // [nm][nq]    basis at volume points (transposed)
  const T* vdphiT;         // [d][nm][nq] physical gradients (transposed)
  const T* vphi;           // [nq][nm]
  const T* vdphi;          // [d][nq][nm]
  const T* vw;             // [nq]        weights * |J|
  const T* fphiT;          // [2d][nm][nqf] traces on local face f = 2k + side
  const T* fdphiT;         // [2d][d][nm][nqf]
  const T* fphi;           // [2d][nqf][nm]
  const T* fdphi;          // [2d][d][nqf][nm]
  const T* fw;             // [d][nqf]    face weights * |J_F|
  const T* lift;           // [2d][nqf q'][nqf q] BR2 lifting operator P[q][q'] (eq. re) incl. 1/(2|J|)
  const T* liftT;          // [2d][2][nqf][nm] lifted test functions of local face f:
                           //   sum_q fw(q) phi_i(q) P[q][q'], P = lift[2k+1] (c=0) or lift[2k] (c=1)
  const T* fpk;            // [2d][nm][nqf][4] (phi_i, d_0 phi_i, .., d_{d-1} phi_i, 0 ..) at face point q
  const T* fpw;            // [2d][nqf][nm][4] the same times the face weight fw(q)
  T detJ;
};

// padded length of a short vector of T in shared memory: a multiple of 16 bytes
__host__ __device__ constexpr int pad16(int n, int size) { return size == 4 ? ((n + 3) & ~3) : ((n + 1) & ~1); }

// N consecutive values from a 16-byte aligned address (N * sizeof(T) a
// multiple of 16): 16-byte loads
template <class T, int N>
__device__ __forceinline__ void ld_vec(const T* p, T* out) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
      const float4 t = reinterpret_cast<const float4*>(p)[k];
      out[4 * k] = t.x;
      out[4 * k + 1] = t.y;
      out[4 * k + 2] = t.z;
      out[4 * k + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const double2 t = reinterpret_cast<const double2*>(p)[k];
      out[2 * k] = t.x;
      out[2 * k + 1] = t.y;
    }
  }
}

}  // namespace dgk
