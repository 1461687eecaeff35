// DG residual and exact Jacobian-vector product kernels (Sec. 3.1 eq. dg_ns with
// the Roe flux, the BR2 viscous flux of eq. visc_flux and the lifting of eq. re;
// Sec. 5.1 eq. ODEDG).
//
// Two kernels per evaluation:
//  face_kernel   one pass over the d*E faces (face (k, e) joins element e, on its
//                xi_k = +1 side, to its +e_k neighbour).  Per face point: traces
//                of u and grad u on both sides, Roe flux, averaged viscous flux,
//                the BR2 lifting of the jump on both sides (a face-point operator
//                applied through shared memory), the dual-consistency tensors.
//                The projections onto both elements' test functions go to face
//                slots [e][k][side][v][i] (no atomics).
//  volume_kernel one pass over the elements: interpolation of u and grad u at the
//                volume points, F_c + F_v, projection onto grad phi_i, then the
//                2d face slots of the element in fixed order (deterministic sums),
//                plus sigma |J| v for a JVP or minus a source for a residual.
// With S = Dual<T> the same code carries the directional derivative: the JVP
// is the exact linearisation of the discrete residual.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <type_traits>

#include "dg_internal.h"

namespace dgk {

template <class T>
__device__ __forceinline__ int dof(int nm, int v, int i) {
  return v * nm + i;
}

// ---------------------------------------------------------------- face kernel
// Shared memory per face (MP = M, DP = M d, each padded to 16 bytes):
//   sW, sV [2][nm][MP]  coefficients of both elements, mode-major (one mode's M
//                       variables in one or two 16-byte loads)
//   sG [2][nqf][MP]     normal column of K(u)(jump n), both sides
//   sF [nqf][MP]        flux (Roe + averaged F_v, + lifting)
//   sD [2][nqf][DP]     dual-consistency tensors / 2, both sides
// The trace tables are packed (phi, grad phi) per mode and point (fpk, and
// fpw with the face weight folded in for the projection), so a mode costs one
// 16-byte table load per side.
template <int D, class T, bool JVP>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 256 : 128, sizeof(T) == 4 ? 2 : 1) face_kernel(MeshView<T> mv, Phys<T> ph,
                                                   const T* __restrict__ W,
                                                   const T* __restrict__ V,
                                                   T* __restrict__ slots, int* status, int fpc,
                                                   const T* __restrict__ Pf) {
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  constexpr int M = D + 2, PU = M * (1 + D);
  constexpr int MP = pad16(M, sizeof(T)), DP = pad16(M * D, sizeof(T));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int nb = mv.nb, nm = mv.nm, nqf = mv.nqf, E = mv.E;
  const int nfaces = D * E;
  const int f0 = blockIdx.x * fpc;
  const int nloc = min(fpc, nfaces - f0);
  if (nloc <= 0) return;
  const size_t cz = (size_t)fpc * 2 * nm * MP;
  T* sW = sm;                                   // [fpc][2][nm][MP]
  T* sV = sW + cz;                              // [fpc][2][nm][MP] (JVP)
  T* sG = sV + (JVP ? cz : 0);                  // [fpc][2][nqf][MP]
  T* sF = sG + (size_t)fpc * 2 * nqf * MP;      // [fpc][nqf][MP]
  T* sD = sF + (size_t)fpc * nqf * MP;          // [fpc][2][nqf][DP]
  // phase 0: stage the modal coefficients of both elements of every face
  for (int t = threadIdx.x; t < nloc * 2 * nb; t += blockDim.x) {
    const int fl = t / (2 * nb), r = t % (2 * nb), side = r / nb, j = r % nb, v = j / nm, i = j % nm;
    const int f = f0 + fl, k = f / E, e = f % E;
    const int el = side == 0 ? e : mv.nbr[(e * D + k) * 2 + 1];
    const size_t o = ((size_t)(fl * 2 + side) * nm + i) * MP + v;
    if (!Pf) sW[o] = W[(size_t)el * nb + j];
    if (JVP) sV[o] = V[(size_t)el * nb + j];
  }
  __syncthreads();
  // phase 1: pointwise physics at the face points (with Pf, a JVP takes the
  // primal traces of both sides from the cache and interpolates only v)
  for (int t = threadIdx.x; t < nloc * nqf; t += blockDim.x) {
    const int fl = t / nqf, q = t % nqf;
    const int f = f0 + fl, k = f / E;
    const int fL = 2 * k + 1, fR = 2 * k;     // local face of L (xi_k = +1) and R (xi_k = -1)
    const T* pkL = mv.fpk + ((size_t)fL * nm * nqf + q) * 4;   // mode i at + i * nqf * 4
    const T* pkR = mv.fpk + ((size_t)fR * nm * nqf + q) * 4;
    const T* wL = sW + (size_t)fl * 2 * nm * MP;
    const T* wR = wL + (size_t)nm * MP;
    const T* vL = sV + (size_t)fl * 2 * nm * MP;
    const T* vR = vL + (size_t)nm * MP;
    S uL[M], uR[M], gL[M][D], gR[M][D];
    bool interp = true;
    if constexpr (JVP) {
      if (Pf) {
        interp = false;
        T tL[M], tR[M], hL[M][D], hR[M][D];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          tL[v] = tR[v] = T(0);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) hL[v][kk] = hR[v][kk] = T(0);
        }
        for (int i = 0; i < nm; ++i) {
          T pL[4], pR[4], a[MP], b[MP];
          ld_vec<T, 4>(pkL + (size_t)i * nqf * 4, pL);
          ld_vec<T, 4>(pkR + (size_t)i * nqf * 4, pR);
          ld_vec<T, MP>(vL + (size_t)i * MP, a);
          ld_vec<T, MP>(vR + (size_t)i * MP, b);
#pragma unroll
          for (int v = 0; v < M; ++v) {
            tL[v] += a[v] * pL[0];
            tR[v] += b[v] * pR[0];
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
              hL[v][kk] += a[v] * pL[1 + kk];
              hR[v][kk] += b[v] * pR[1 + kk];
            }
          }
        }
        const T* cL = Pf + ((size_t)(f0 + fl) * nqf + q) * 2 * PU;
        const T* cR = cL + PU;
#pragma unroll
        for (int v = 0; v < M; ++v) {
          uL[v] = S(cL[v], tL[v]);
          uR[v] = S(cR[v], tR[v]);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) {
            gL[v][kk] = S(cL[M + v * D + kk], hL[v][kk]);
            gR[v][kk] = S(cR[M + v * D + kk], hR[v][kk]);
          }
        }
      }
    }
    if (interp) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        uL[v] = T(0);
        uR[v] = T(0);
#pragma unroll
        for (int kk = 0; kk < D; ++kk) {
          gL[v][kk] = T(0);
          gR[v][kk] = T(0);
        }
      }
      for (int i = 0; i < nm; ++i) {
        T pL[4], pR[4], a0[MP], b0[MP];
        ld_vec<T, 4>(pkL + (size_t)i * nqf * 4, pL);
        ld_vec<T, 4>(pkR + (size_t)i * nqf * 4, pR);
        ld_vec<T, MP>(wL + (size_t)i * MP, a0);
        ld_vec<T, MP>(wR + (size_t)i * MP, b0);
        T a1[MP], b1[MP];
        if constexpr (JVP) {
          ld_vec<T, MP>(vL + (size_t)i * MP, a1);
          ld_vec<T, MP>(vR + (size_t)i * MP, b1);
        }
#pragma unroll
        for (int v = 0; v < M; ++v) {
          S a, b;
          if constexpr (JVP) {
            a = S(a0[v], a1[v]);
            b = S(b0[v], b1[v]);
          } else {
            a = a0[v];
            b = b0[v];
          }
          uL[v] = uL[v] + a * pL[0];
          uR[v] = uR[v] + b * pR[0];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) {
            gL[v][kk] = gL[v][kk] + a * pL[1 + kk];
            gR[v][kk] = gR[v][kk] + b * pR[1 + kk];
          }
        }
      }
    }
    if (!physical<D>(uL, ph.gm1) || !physical<D>(uR, ph.gm1))
      atomicOr(status, ST_NONPHYSICAL);
    S fp[M], GLn[M], GRn[M], DL[M][D], DR[M][D];
    face_point_k<D, S, T>(k, uL, gL, uR, gR, ph, fp, GLn, GRn, DL, DR);
    T* g0 = sG + ((size_t)fl * 2 * nqf + q) * MP;
    T* g1 = sG + ((size_t)(fl * 2 + 1) * nqf + q) * MP;
    T* fo = sF + ((size_t)fl * nqf + q) * MP;
    T* d0 = sD + (((size_t)fl * 2) * nqf + q) * DP;
    T* d1 = sD + (((size_t)fl * 2 + 1) * nqf + q) * DP;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      fo[v] = JVP ? tan_part(fp[v]) : val(fp[v]);
      g0[v] = JVP ? tan_part(GLn[v]) : val(GLn[v]);
      g1[v] = JVP ? tan_part(GRn[v]) : val(GRn[v]);
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        d0[v * D + kk] = JVP ? tan_part(DL[v][kk]) : val(DL[v][kk]);
        d1[v * D + kk] = JVP ? tan_part(DR[v][kk]) : val(DR[v][kk]);
      }
    }
  }
  __syncthreads();
  // phase 2: BR2 lifting on both sides, fhat = Roe + {F_v}.n + eta {delta}.n
  for (int t = threadIdx.x; t < nloc * nqf; t += blockDim.x) {
    const int fl = t / nqf, q = t % nqf;
    const int k = (f0 + fl) / E;
    const T* PL = mv.lift + (size_t)(2 * k + 1) * nqf * nqf + q;   // column q2 at PL[q2 * nqf]
    const T* PR = mv.lift + (size_t)(2 * k) * nqf * nqf + q;
    const T* gA = sG + (size_t)fl * 2 * nqf * MP;
    const T* gB = gA + (size_t)nqf * MP;
    T dl[M], dr[M];
#pragma unroll
    for (int v = 0; v < M; ++v) dl[v] = dr[v] = T(0);
    for (int q2 = 0; q2 < nqf; ++q2) {
      const T a = PL[(size_t)q2 * nqf], b = PR[(size_t)q2 * nqf];
      T ga[MP], gb[MP];
      ld_vec<T, MP>(gA + (size_t)q2 * MP, ga);
      ld_vec<T, MP>(gB + (size_t)q2 * MP, gb);
#pragma unroll
      for (int v = 0; v < M; ++v) {
        dl[v] += a * ga[v];
        dr[v] += b * gb[v];
      }
    }
    T* fo = sF + ((size_t)fl * nqf + q) * MP;
#pragma unroll
    for (int v = 0; v < M; ++v) fo[v] += ph.eta * T(0.5) * (dl[v] + dr[v]);
  }
  __syncthreads();
  // phase 3: projection onto the test functions of both elements, a thread per
  // (face, side, mode) and all M variables
  for (int t = threadIdx.x; t < nloc * 2 * nm; t += blockDim.x) {
    const int fl = t / (2 * nm), r = t % (2 * nm), side = r / nm, i = r % nm;
    const int f = f0 + fl, k = f / E, e = f % E;
    const int lf = side == 0 ? 2 * k + 1 : 2 * k;
    const T sgn = side == 0 ? T(1) : T(-1);
    const T* pw = mv.fpw + ((size_t)lf * nqf * nm + i) * 4;   // point q at + q * nm * 4
    const T* Fo = sF + (size_t)fl * nqf * MP;
    const T* Dd = sD + (size_t)(fl * 2 + side) * nqf * DP;
    T acc[M];
#pragma unroll
    for (int v = 0; v < M; ++v) acc[v] = T(0);
    for (int q = 0; q < nqf; ++q) {
      T w4[4], fq[MP], dq[DP];
      ld_vec<T, 4>(pw + (size_t)q * nm * 4, w4);
      ld_vec<T, MP>(Fo + (size_t)q * MP, fq);
      ld_vec<T, DP>(Dd + (size_t)q * DP, dq);
      const T sw = sgn * w4[0];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        T s_ = sw * fq[v];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) s_ -= w4[1 + kk] * dq[v * D + kk];
        acc[v] += s_;
      }
    }
    T* out = slots + (((size_t)e * D + k) * 2 + side) * nb + i;
#pragma unroll
    for (int v = 0; v < M; ++v) out[(size_t)v * nm] = acc[v];
  }
}

// ---------------------------------------------------------------- volume kernel
template <int D, class T, bool JVP>
__global__ void __launch_bounds__(256) volume_kernel(MeshView<T> mv, Phys<T> ph,
                                                     const T* __restrict__ W,
                                                     const T* __restrict__ V,
                                                     const T* __restrict__ slots,
                                                     const T* __restrict__ Src, T sigma,
                                                     T* __restrict__ out, int* status, int epc) {
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  constexpr int M = D + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, E = mv.E;
  const int e0 = blockIdx.x * epc;
  const int nloc = min(epc, E - e0);
  if (nloc <= 0) return;
  T* sW = sm;                                  // [epc][nb]
  T* sV = sW + (size_t)epc * nb;               // [epc][nb]
  T* sF = sV + (JVP ? (size_t)epc * nb : 0);   // [epc][nq][M][D]  w_q |J| F
  for (int t = threadIdx.x; t < nloc * nb; t += blockDim.x) {
    sW[t] = W[(size_t)e0 * nb + t];
    if (JVP) sV[t] = V[(size_t)e0 * nb + t];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nloc * nq; t += blockDim.x) {
    int el = t / nq, q = t % nq;
    const T* w = sW + (size_t)el * nb;
    const T* vv = sV + (size_t)el * nb;
    S u[M], g[M][D];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      u[v] = T(0);
#pragma unroll
      for (int kk = 0; kk < D; ++kk) g[v][kk] = T(0);
    }
    for (int i = 0; i < nm; ++i) {
      T p = mv.vphiT[(size_t)i * nq + q];
      T dp[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) dp[kk] = mv.vdphiT[((size_t)kk * nm + i) * nq + q];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        S a;
        if constexpr (JVP) a = S(w[v * nm + i], vv[v * nm + i]);
        else a = w[v * nm + i];
        u[v] = u[v] + a * p;
#pragma unroll
        for (int kk = 0; kk < D; ++kk) g[v][kk] = g[v][kk] + a * dp[kk];
      }
    }
    if (!physical<D>(u, ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
    S F[M][D];
    flux_total<D, S, T>(u, g, F, ph);
    T wq = mv.vw[q];
    T* fo = sF + ((size_t)el * nq + q) * M * D;
#pragma unroll
    for (int v = 0; v < M; ++v)
#pragma unroll
      for (int kk = 0; kk < D; ++kk) fo[v * D + kk] = wq * (JVP ? tan_part(F[v][kk]) : val(F[v][kk]));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nloc * nb; t += blockDim.x) {
    int el = t / nb, j = t % nb;
    int v = j / nm, i = j % nm;
    int e = e0 + el;
    const T* fo = sF + (size_t)el * nq * M * D;
    T acc = T(0);
    for (int q = 0; q < nq; ++q) {
      const T* fq = fo + (size_t)q * M * D + v * D;
#pragma unroll
      for (int kk = 0; kk < D; ++kk) acc -= mv.vdphi[((size_t)kk * nq + q) * nm + i] * fq[kk];
    }
    // face contributions in fixed order: for each direction, own +k face then -k face
#pragma unroll
    for (int k = 0; k < D; ++k) {
      int em = mv.nbr[(e * D + k) * 2 + 0];
      acc += slots[(((size_t)e * D + k) * 2 + 0) * nb + j];
      acc += slots[(((size_t)em * D + k) * 2 + 1) * nb + j];
    }
    if (JVP) acc += sigma * mv.detJ * sV[t];
    else if (Src) acc -= Src[(size_t)e * nb + j];
    out[(size_t)e * nb + j] = acc;
  }
}

// FP32 volume kernel with the basis tables in shared memory: one persistent
// CTA per SM stages Tab[0][i][q] = phi_i(q) and Tab[1+k][i][q] = d phi_i/dx_k (q)
// once (q padded to an odd stride, so that the column reads are free of bank
// conflicts), then NSLOT independent groups of 256 threads each walk over
// elements, synchronising only among themselves (named barriers).  The same
// three phases as volume_kernel: interpolation (thread per point, the
// coefficients mode-major so that one mode's M variables are two 16-byte
// loads), F_c + F_v (a point's M x D values padded to FP for 16-byte loads),
// and the projection, where a thread takes one mode i and every NC-th point
// for all M variables (the point's fluxes read once for M outputs); the NC
// partial sums of each output are added in a fixed order, with the face slots.
template <int D, bool JVP, int NSLOT>
__global__ void __launch_bounds__(256 * NSLOT, 1) volume_kernel_st(MeshView<float> mv, Phys<float> ph,
                                                                   const float* __restrict__ W,
                                                                   const float* __restrict__ V,
                                                                   const float* __restrict__ slots,
                                                                   const float* __restrict__ Src, float sigma,
                                                                   float* __restrict__ out, int* status,
                                                                   int nqp, const float* __restrict__ Pv) {
  using T = float;
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  constexpr int M = D + 2, NT = 1 + D, PU = M * (1 + D);
  constexpr int MP = pad16(M, 4), FP = pad16(M * D, 4);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, E = mv.E;
  T* Tab = reinterpret_cast<T*>(smem_raw);            // [1 + D][nm][nqp]
  T* sw = Tab + (size_t)NT * nm * nqp;                 // [nq] weights * |J|
  const size_t per_slot = (size_t)nm * MP * (JVP ? 2 : 1) + (size_t)nq * FP;
  for (int t = threadIdx.x; t < NT * nm * nq; t += blockDim.x) {
    const int r = t / nq, q = t - r * nq;               // r = kk * nm + i
    const int kk = r / nm, i = r - kk * nm;
    Tab[(size_t)r * nqp + q] = kk == 0 ? mv.vphiT[(size_t)i * nq + q]
                                       : mv.vdphiT[((size_t)(kk - 1) * nm + i) * nq + q];
  }
  for (int t = threadIdx.x; t < nq; t += blockDim.x) sw[t] = mv.vw[t];
  __syncthreads();
  const int slot = threadIdx.x >> 8, tid = threadIdx.x & 255;
  T* sW = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(sw + nq) + 15) & ~uintptr_t(15)) +
       (size_t)slot * ((per_slot + 3) / 4 * 4);
  T* sV = sW + (size_t)nm * MP;                         // [nm][MP]
  T* sF = sV + (JVP ? (size_t)nm * MP : 0);             // [nq][FP]; then the projection's partial sums
  // projection split: NC point classes per mode, the partials [NC][nb] fit in sF
  const int NC = max(1, min(min(256 / nm, nq), (int)(((size_t)nq * FP) / nb)));
  const int bar = 1 + slot;
  for (int e = blockIdx.x * NSLOT + slot; e < E; e += gridDim.x * NSLOT) {
    for (int t = tid; t < nb; t += 256) {
      const int v = t / nm, i = t - v * nm;
      if (!Pv) sW[i * MP + v] = W[(size_t)e * nb + t];
      if (JVP) sV[i * MP + v] = V[(size_t)e * nb + t];
    }
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
    for (int q = tid; q < nq; q += 256) {
      S u[M], g[M][D];
      const T* tq = Tab + q;
      bool interp = true;
      if constexpr (JVP) {
        if (Pv) {   // primal traces from the cache, interpolate only v
          interp = false;
          T tv[M], th[M][D];
#pragma unroll
          for (int v = 0; v < M; ++v) {
            tv[v] = T(0);
#pragma unroll
            for (int kk = 0; kk < D; ++kk) th[v][kk] = T(0);
          }
          for (int i = 0; i < nm; ++i) {
            const T p = tq[(size_t)i * nqp];
            T dp[D], a[MP];
#pragma unroll
            for (int kk = 0; kk < D; ++kk) dp[kk] = tq[((size_t)(1 + kk) * nm + i) * nqp];
            ld_vec<T, MP>(sV + (size_t)i * MP, a);
#pragma unroll
            for (int v = 0; v < M; ++v) {
              tv[v] += a[v] * p;
#pragma unroll
              for (int kk = 0; kk < D; ++kk) th[v][kk] += a[v] * dp[kk];
            }
          }
          const T* c = Pv + ((size_t)e * nq + q) * PU;
#pragma unroll
          for (int v = 0; v < M; ++v) {
            u[v] = S(c[v], tv[v]);
#pragma unroll
            for (int kk = 0; kk < D; ++kk) g[v][kk] = S(c[M + v * D + kk], th[v][kk]);
          }
        }
      }
      if (interp) {
#pragma unroll
        for (int v = 0; v < M; ++v) {
          u[v] = T(0);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) g[v][kk] = T(0);
        }
        for (int i = 0; i < nm; ++i) {
          const T p = tq[(size_t)i * nqp];
          T dp[D], a0[MP], a1[MP];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) dp[kk] = tq[((size_t)(1 + kk) * nm + i) * nqp];
          ld_vec<T, MP>(sW + (size_t)i * MP, a0);
          if constexpr (JVP) ld_vec<T, MP>(sV + (size_t)i * MP, a1);
#pragma unroll
          for (int v = 0; v < M; ++v) {
            S a;
            if constexpr (JVP) a = S(a0[v], a1[v]);
            else a = a0[v];
            u[v] = u[v] + a * p;
#pragma unroll
            for (int kk = 0; kk < D; ++kk) g[v][kk] = g[v][kk] + a * dp[kk];
          }
        }
      }
      if (!physical<D>(u, ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
      S F[M][D];
      flux_total<D, S, T>(u, g, F, ph);
      const T wq = sw[q];
      T* fo = sF + (size_t)q * FP;
#pragma unroll
      for (int v = 0; v < M; ++v)
#pragma unroll
        for (int kk = 0; kk < D; ++kk) fo[v * D + kk] = wq * (JVP ? tan_part(F[v][kk]) : val(F[v][kk]));
    }
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
    // projection onto grad phi_i: partial sums over the points q = c, c + NC, ..
    T acc[M];
    const int pi = tid % nm, pc = tid / nm;
    if (pc < NC) {
#pragma unroll
      for (int v = 0; v < M; ++v) acc[v] = T(0);
      for (int q = pc; q < nq; q += NC) {
        T dp[D], f[FP];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) dp[kk] = Tab[((size_t)(1 + kk) * nm + pi) * nqp + q];
        ld_vec<T, FP>(sF + (size_t)q * FP, f);
#pragma unroll
        for (int v = 0; v < M; ++v)
#pragma unroll
          for (int kk = 0; kk < D; ++kk) acc[v] += dp[kk] * f[v * D + kk];
      }
    }
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
    if (pc < NC) {
#pragma unroll
      for (int v = 0; v < M; ++v) sF[(size_t)pc * nb + v * nm + pi] = acc[v];
    }
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
    for (int j = tid; j < nb; j += 256) {
      T a = T(0);
      for (int c = 0; c < NC; ++c) a -= sF[(size_t)c * nb + j];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int em = mv.nbr[(e * D + k) * 2 + 0];
        a += slots[(((size_t)e * D + k) * 2 + 0) * nb + j];
        a += slots[(((size_t)em * D + k) * 2 + 1) * nb + j];
      }
      if (JVP) a += sigma * mv.detJ * sV[(j % nm) * MP + j / nm];
      else if (Src) a -= Src[(size_t)e * nb + j];
      out[(size_t)e * nb + j] = a;
    }
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
  }
}

constexpr int VOL_SLOTS = 3;

// Shared memory of volume_kernel_st (FP32), when the tables fit beside the slots.
static bool vol_tables_fit(const Mesh& M, bool jvp, size_t* bytes, int* nqp) {
  if (M.nb > 256) return false;
  *nqp = M.nq | 1;
  const size_t per_slot = (size_t)M.nm * pad16(M.m, 4) * (jvp ? 2 : 1) + (size_t)M.nq * pad16(M.m * M.d, 4);
  const size_t n = (size_t)(1 + M.d) * M.nm * *nqp + M.nq;
  *bytes = n * sizeof(float) + 16 + VOL_SLOTS * ((per_slot + 3) / 4 * 4) * sizeof(float);
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return *bytes <= (size_t)smax;
}

template <class T>
static size_t face_smem(const Mesh& M, int fpc, bool jvp) {
  const size_t MP = pad16(M.m, sizeof(T)), DP = pad16(M.m * M.d, sizeof(T));
  return sizeof(T) * (size_t)fpc * (2 * M.nm * MP * (jvp ? 2 : 1) + 2 * M.nqf * MP + M.nqf * MP + 2 * M.nqf * DP);
}
template <class T>
static size_t vol_smem(const Mesh& M, int epc, bool jvp) {
  return sizeof(T) * (size_t)epc * (M.nb * (jvp ? 2 : 1) + M.nq * M.m * M.d);
}

template <int D, class T, bool JVP>
static cudaError_t run_residual(const Mesh& Ms, const T* W, const T* V, const T* S, T sigma, T* out,
                                cudaStream_t st, const T* Pv, const T* Pf, int parts) {
  MeshView<T> mv = Ms.view<T>();
  Phys<T> ph = Ms.phys_t<T>();
  T* slots = std::is_same<T, double>::value ? (T*)Ms.t64.slots : (T*)Ms.t32.slots;
  // FP32: 256 threads over 256 / n_qf faces (7 at p = 4: 252 of 256 threads busy per point
  // phase, against 108 of 128 with 3 faces), two CTAs per SM at 128 registers, when two
  // such CTAs fit shared memory (not for the 125 modes of Q_4: then 128 threads)
  int fthreads = 128;
  if (sizeof(T) == 4 && face_smem<T>(Ms, std::max(1, 256 / Ms.nqf), JVP) <= 100 * 1024) fthreads = 256;
  int fpc = std::max(1, fthreads / Ms.nqf);
  size_t fsm = face_smem<T>(Ms, fpc, JVP);
  while (fsm > 200 * 1024 && fpc > 1) fsm = face_smem<T>(Ms, --fpc, JVP);
  if (fsm > 48 * 1024)
    allow_max_smem(face_kernel<D, T, JVP>);
  int nfaces = D * Ms.E;
  if (parts & 1) {
    // 3-D: the face term by sum factorisation in FP64 (fewer of the FP64 pipe's
    // cycles: the residual 4.4 -> 3.8 ms at 16^3 p = 4, 125 -> 73 ms at 32^3
    // p = 6); in FP32 the direct kernel is faster (smoother JVP 0.23 against
    // 0.56 ms at p = 4, 4.9 against 9.1 ms at p = 6).  DG_NO_SUMFACT_FACE=1
    // keeps the direct kernel; DG_SUMFACT_FACE_MIN_MODES=n takes the sum-
    // factorised one in FP32 from n modes on
    const char* nsff = getenv("DG_NO_SUMFACT_FACE");
    const char* sfmin = getenv("DG_SUMFACT_FACE_MIN_MODES");
    const int min_modes = sfmin ? atoi(sfmin) : INT_MAX;
    cudaError_t e = cudaErrorNotSupported;
    if (D == 3 && !(nsff && nsff[0] == '1') && (std::is_same<T, double>::value || Ms.nm >= min_modes)) {
      e = launch_face_sf<T>(Ms, W, V, slots, JVP, JVP ? Pf : nullptr, st);
      if (e == cudaErrorNotSupported) (void)cudaGetLastError();
    }
    if (e == cudaErrorNotSupported) {
      note_launch();
      face_kernel<D, T, JVP><<<(nfaces + fpc - 1) / fpc, fthreads, fsm, st>>>(mv, ph, W, V, slots, Ms.status, fpc,
                                                                        JVP ? Pf : nullptr);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
  }
  if (!(parts & 2)) return cudaSuccess;
  // volume term by sum factorisation (Q_p; P_p embedded in Q_p, 3-D) when its
  // stages fit shared memory, except in FP32 where the shared-memory kernel's
  // tables fit (it reads the cached primal traces and interpolates only the
  // direction); DG_NO_SUMFACT_P=1 keeps the direct kernels for P_p
  size_t tsm0 = 0;
  int nqp0 = 0;
  const bool st_fits = std::is_same<T, float>::value && vol_tables_fit(Ms, JVP, &tsm0, &nqp0);
  const char* nsf = getenv("DG_NO_SUMFACT_P");
  const bool sumfact = Ms.desc.space == DG_SPACE_Q || (!(nsf && nsf[0] == '1') && !st_fits && Ms.d == 3);
  if (sumfact) {
    cudaError_t eq = launch_volume_q<T>(Ms, W, V, S, sigma, JVP, out, st);
    if (eq != cudaErrorNotSupported) return eq;
    (void)cudaGetLastError();
  }
  if constexpr (std::is_same<T, float>::value) {
    size_t tsm;
    int nqp;
    if (vol_tables_fit(Ms, JVP, &tsm, &nqp)) {
      allow_max_smem(volume_kernel_st<D, JVP, VOL_SLOTS>);
      int dev = 0, nsm = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      const int grid = std::min(nsm, (Ms.E + VOL_SLOTS - 1) / VOL_SLOTS);
      note_launch();
      volume_kernel_st<D, JVP, VOL_SLOTS><<<grid, 256 * VOL_SLOTS, tsm, st>>>(mv, ph, W, V, slots, S, sigma, out,
                                                                             Ms.status, nqp,
                                                                             JVP ? (const float*)Pv : nullptr);
      return cudaGetLastError();
    }
  }
  int epc = std::max(1, 256 / Ms.nq);
  size_t vsm = vol_smem<T>(Ms, epc, JVP);
  while (vsm > 200 * 1024 && epc > 1) vsm = vol_smem<T>(Ms, --epc, JVP);
  if (vsm > 48 * 1024)
    allow_max_smem(volume_kernel<D, T, JVP>);
  note_launch();
  volume_kernel<D, T, JVP><<<(Ms.E + epc - 1) / epc, 256, vsm, st>>>(mv, ph, W, V, slots, S, sigma, out,
                                                                    Ms.status, epc);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_residual(const Mesh& M, const T* W, const T* V, const T* S, T sigma, bool jvp, T* out,
                            cudaStream_t st, const T* Pv, const T* Pf, int parts) {
  if (M.kind == DG_MESH_TRI) return launch_residual_tri<T>(M, W, V, S, sigma, jvp, out, st);
  if (M.d == 2)
    return jvp ? run_residual<2, T, true>(M, W, V, S, sigma, out, st, Pv, Pf, parts)
               : run_residual<2, T, false>(M, W, V, S, sigma, out, st, nullptr, nullptr, parts);
  return jvp ? run_residual<3, T, true>(M, W, V, S, sigma, out, st, Pv, Pf, parts)
             : run_residual<3, T, false>(M, W, V, S, sigma, out, st, nullptr, nullptr, parts);
}

template cudaError_t launch_residual<double>(const Mesh&, const double*, const double*, const double*, double,
                                             bool, double*, cudaStream_t, const double*, const double*, int);
template cudaError_t launch_residual<float>(const Mesh&, const float*, const float*, const float*, float, bool,
                                            float*, cudaStream_t, const float*, const float*, int);

// Primal traces of the FP32 state at every volume point, Pv[e][q] = (u, grad u),
// and at every face point on both sides, Pf[f][q][side] (face f = k E + e joins
// e, on its xi_k = +1 side, to its +e_k neighbour), in the mode order of the
// kernels' own interpolation.  Computed once per preconditioner refresh: the
// smoother's JVPs then interpolate only their direction.
template <int D>
__global__ void primal_cache_kernel(MeshView<float> mv, const float* __restrict__ W, float* __restrict__ Pv,
                                    float* __restrict__ Pf) {
  constexpr int M = D + 2, PU = M * (1 + D);
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, nqf = mv.nqf, E = mv.E;
  const long nvol = (long)E * nq, nface = (long)D * E * nqf * 2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nvol + nface; t += (long)gridDim.x * blockDim.x) {
    float u[M], g[M][D];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      u[v] = 0.f;
#pragma unroll
      for (int kk = 0; kk < D; ++kk) g[v][kk] = 0.f;
    }
    float* dst;
    if (t < nvol) {
      const long e = t / nq;
      const int q = (int)(t - e * nq);
      const float* w = W + (size_t)e * nb;
      for (int i = 0; i < nm; ++i) {
        const float p = mv.vphiT[(size_t)i * nq + q];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          const float a = w[v * nm + i];
          u[v] += a * p;
#pragma unroll
          for (int kk = 0; kk < D; ++kk) g[v][kk] += a * mv.vdphiT[((size_t)kk * nm + i) * nq + q];
        }
      }
      dst = Pv + (size_t)t * PU;
    } else {
      const long r = t - nvol;
      const int side = (int)(r & 1);
      const long fq = r >> 1, f = fq / nqf;
      const int q = (int)(fq - f * nqf), k = (int)(f / E);
      const long e = f - (long)k * E;
      const long el = side == 0 ? e : mv.nbr[(e * D + k) * 2 + 1];
      const int lf = side == 0 ? 2 * k + 1 : 2 * k;
      const float* w = W + (size_t)el * nb;
      for (int i = 0; i < nm; ++i) {
        const float p = mv.fphiT[((size_t)lf * nm + i) * nqf + q];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          const float a = w[v * nm + i];
          u[v] += a * p;
#pragma unroll
          for (int kk = 0; kk < D; ++kk) g[v][kk] += a * mv.fdphiT[(((size_t)lf * D + kk) * nm + i) * nqf + q];
        }
      }
      dst = Pf + (size_t)r * PU;
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
      dst[v] = u[v];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) dst[M + v * D + kk] = g[v][kk];
    }
  }
}

size_t primal_cache_sizes(const Mesh& M, size_t* nface) {
  const size_t pu = (size_t)M.m * (1 + M.d);
  *nface = (size_t)M.d * M.E * M.nqf * 2 * pu;
  return (size_t)M.E * M.nq * pu;
}

cudaError_t launch_primal_cache(const Mesh& M, const float* W, float* Pv, float* Pf, cudaStream_t st) {
  const long tot = (long)M.E * M.nq + (long)M.d * M.E * M.nqf * 2;
  const int grid = (int)std::min<long>((tot + 255) / 256, 65535L * 4);
  note_launch();
  if (M.d == 2)
    primal_cache_kernel<2><<<grid, 256, 0, st>>>(M.view<float>(), W, Pv, Pf);
  else
    primal_cache_kernel<3><<<grid, 256, 0, st>>>(M.view<float>(), W, Pv, Pf);
  return cudaGetLastError();
}

// FP64 residual with caller-provided face slots (E * d * 2 * nb doubles) in
// place of the mesh handle's own: the same two kernels, launched the same way.
template <int D>
static cudaError_t run_residual_slots(const Mesh& Ms, const double* W, const double* S, double* out,
                                      double* slots, cudaStream_t st) {
  MeshView<double> mv = Ms.view<double>();
  Phys<double> ph = Ms.phys_t<double>();
  int fpc = std::max(1, 128 / Ms.nqf);
  size_t fsm = face_smem<double>(Ms, fpc, false);
  while (fsm > 200 * 1024 && fpc > 1) fsm = face_smem<double>(Ms, --fpc, false);
  if (fsm > 48 * 1024)
    allow_max_smem(face_kernel<D, double, false>);
  int nfaces = D * Ms.E;
  note_launch();
  face_kernel<D, double, false><<<(nfaces + fpc - 1) / fpc, 128, fsm, st>>>(mv, ph, W, nullptr, slots,
                                                                            Ms.status, fpc, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int epc = std::max(1, 256 / Ms.nq);
  size_t vsm = vol_smem<double>(Ms, epc, false);
  while (vsm > 200 * 1024 && epc > 1) vsm = vol_smem<double>(Ms, --epc, false);
  if (vsm > 48 * 1024)
    allow_max_smem(volume_kernel<D, double, false>);
  note_launch();
  volume_kernel<D, double, false><<<(Ms.E + epc - 1) / epc, 256, vsm, st>>>(mv, ph, W, nullptr, slots, S, 0.0,
                                                                           out, Ms.status, epc);
  return cudaGetLastError();
}

cudaError_t launch_residual_with_slots(const Mesh& M, const double* W, const double* S, double* out,
                                       double* slots, cudaStream_t st) {
  return M.d == 2 ? run_residual_slots<2>(M, W, S, out, slots, st) : run_residual_slots<3>(M, W, S, out, slots, st);
}

}  // namespace dgk
