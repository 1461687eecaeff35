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
#include <cstdlib>
#include <type_traits>

#include "dg_internal.h"

namespace dgk {

template <class T>
__device__ __forceinline__ int dof(int nm, int v, int i) {
  return v * nm + i;
}

// ---------------------------------------------------------------- face kernel
template <int D, class T, bool JVP>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) face_kernel(MeshView<T> mv, Phys<T> ph,
                                                   const T* __restrict__ W,
                                                   const T* __restrict__ V,
                                                   T* __restrict__ slots, int* status, int fpc,
                                                   const T* __restrict__ Pf) {
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  constexpr int M = D + 2, PU = M * (1 + D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int nb = mv.nb, nm = mv.nm, nqf = mv.nqf, E = mv.E;
  const int nfaces = D * E;
  const int f0 = blockIdx.x * fpc;
  const int nloc = min(fpc, nfaces - f0);
  if (nloc <= 0) return;
  // shared layout
  T* sW = sm;                                   // [fpc][2][nb]
  T* sV = sW + (size_t)fpc * 2 * nb;            // [fpc][2][nb] (JVP)
  T* sG = sV + (JVP ? (size_t)fpc * 2 * nb : 0);// [fpc][2][nqf][M]  normal column of K(u)(jump n)
  T* sF = sG + (size_t)fpc * 2 * nqf * M;       // [fpc][nqf][M]     flux (Roe + avg F_v, + lifting)
  T* sD = sF + (size_t)fpc * nqf * M;           // [fpc][2][nqf][M][D]  dual tensors / 2
  // phase 0: stage the modal coefficients of both elements of every face
  for (int t = threadIdx.x; t < nloc * 2 * nb; t += blockDim.x) {
    int fl = t / (2 * nb), r = t % (2 * nb), side = r / nb, j = r % nb;
    int f = f0 + fl, k = f / E, e = f % E;
    int el = side == 0 ? e : mv.nbr[(e * D + k) * 2 + 1];
    if (!Pf) sW[t] = W[(size_t)el * nb + j];
    if (JVP) sV[t] = V[(size_t)el * nb + j];
  }
  __syncthreads();
  // phase 1: pointwise physics at the face points (with Pf, a JVP takes the
  // primal traces of both sides from the cache and interpolates only v)
  for (int t = threadIdx.x; t < nloc * nqf; t += blockDim.x) {
    int fl = t / nqf, q = t % nqf;
    int f = f0 + fl, k = f / E;
    int fL = 2 * k + 1, fR = 2 * k;           // local face of L (xi_k = +1) and R (xi_k = -1)
    S uL[M], uR[M], gL[M][D], gR[M][D];
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
    const T* wL = sW + (size_t)fl * 2 * nb;
    const T* wR = wL + nb;
    const T* vL = sV + (size_t)fl * 2 * nb;
    const T* vR = vL + nb;
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
          const T pL = mv.fphiT[((size_t)fL * nm + i) * nqf + q];
          const T pR = mv.fphiT[((size_t)fR * nm + i) * nqf + q];
          T dL[D], dR[D];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) {
            dL[kk] = mv.fdphiT[(((size_t)fL * D + kk) * nm + i) * nqf + q];
            dR[kk] = mv.fdphiT[(((size_t)fR * D + kk) * nm + i) * nqf + q];
          }
#pragma unroll
          for (int v = 0; v < M; ++v) {
            const T a = vL[v * nm + i], b = vR[v * nm + i];
            tL[v] += a * pL;
            tR[v] += b * pR;
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
              hL[v][kk] += a * dL[kk];
              hR[v][kk] += b * dR[kk];
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
    for (int i = 0; interp && i < nm; ++i) {
      T pL = mv.fphiT[((size_t)fL * nm + i) * nqf + q];
      T pR = mv.fphiT[((size_t)fR * nm + i) * nqf + q];
      T dL[D], dR[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        dL[kk] = mv.fdphiT[(((size_t)fL * D + kk) * nm + i) * nqf + q];
        dR[kk] = mv.fdphiT[(((size_t)fR * D + kk) * nm + i) * nqf + q];
      }
#pragma unroll
      for (int v = 0; v < M; ++v) {
        S a, b;
        if constexpr (JVP) {
          a = S(wL[v * nm + i], vL[v * nm + i]);
          b = S(wR[v * nm + i], vR[v * nm + i]);
        } else {
          a = wL[v * nm + i];
          b = wR[v * nm + i];
        }
        uL[v] = uL[v] + a * pL;
        uR[v] = uR[v] + b * pR;
#pragma unroll
        for (int kk = 0; kk < D; ++kk) {
          gL[v][kk] = gL[v][kk] + a * dL[kk];
          gR[v][kk] = gR[v][kk] + b * dR[kk];
        }
      }
    }
    if (!physical<D>(uL, ph.gm1) || !physical<D>(uR, ph.gm1))
      atomicOr(status, ST_NONPHYSICAL);
    S fp[M], GLn[M], GRn[M], DL[M][D], DR[M][D];
    face_point_k<D, S, T>(k, uL, gL, uR, gR, ph, fp, GLn, GRn, DL, DR);
    T* g0 = sG + ((size_t)fl * 2 * nqf + q) * M;
    T* g1 = sG + ((size_t)(fl * 2 + 1) * nqf + q) * M;
    T* fo = sF + ((size_t)fl * nqf + q) * M;
    T* d0 = sD + (((size_t)fl * 2) * nqf + q) * M * D;
    T* d1 = sD + (((size_t)fl * 2 + 1) * nqf + q) * M * D;
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
    int fl = t / nqf, q = t % nqf;
    int k = (f0 + fl) / E;
    const T* PL = mv.lift + ((size_t)(2 * k + 1) * nqf + q) * nqf;
    const T* PR = mv.lift + ((size_t)(2 * k) * nqf + q) * nqf;
    T dl[M], dr[M];
#pragma unroll
    for (int v = 0; v < M; ++v) dl[v] = dr[v] = T(0);
    for (int q2 = 0; q2 < nqf; ++q2) {
      T a = PL[q2], b = PR[q2];
      const T* g0 = sG + ((size_t)fl * 2 * nqf + q2) * M;
      const T* g1 = sG + ((size_t)(fl * 2 + 1) * nqf + q2) * M;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        dl[v] += a * g0[v];
        dr[v] += b * g1[v];
      }
    }
    T* fo = sF + ((size_t)fl * nqf + q) * M;
#pragma unroll
    for (int v = 0; v < M; ++v) fo[v] += ph.eta * T(0.5) * (dl[v] + dr[v]);
  }
  __syncthreads();
  // phase 3: projection onto the test functions of both elements
  for (int t = threadIdx.x; t < nloc * 2 * nb; t += blockDim.x) {
    int fl = t / (2 * nb), r = t % (2 * nb), side = r / nb, j = r % nb;
    int v = j / nm, i = j % nm;
    int f = f0 + fl, k = f / E, e = f % E;
    int lf = side == 0 ? 2 * k + 1 : 2 * k;
    T sgn = side == 0 ? T(1) : T(-1);
    const T* fw = mv.fw + (size_t)k * nqf;
    const T* ph_ = mv.fphi + (size_t)lf * nqf * nm;
    const T* dph = mv.fdphi + (size_t)lf * D * nqf * nm;
    const T* Fo = sF + (size_t)fl * nqf * M;
    const T* Dd = sD + ((size_t)(fl * 2 + side) * nqf) * M * D;
    T acc = T(0);
    for (int q = 0; q < nqf; ++q) {
      T s = sgn * ph_[(size_t)q * nm + i] * Fo[q * M + v];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) s -= dph[((size_t)kk * nqf + q) * nm + i] * Dd[(q * M + v) * D + kk];
      acc += fw[q] * s;
    }
    slots[(((size_t)e * D + k) * 2 + side) * nb + j] = acc;
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
// once (q padded to an odd stride, so that the projection's column reads are
// free of bank conflicts), then NSLOT independent groups of 256 threads each
// walk over elements, synchronising only among themselves (named barriers).
// The same three phases as volume_kernel: interpolation (thread per point),
// F_c + F_v, projection (thread per (v, i)) plus the face slots.
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, E = mv.E;
  T* Tab = reinterpret_cast<T*>(smem_raw);            // [1 + D][nm][nqp]
  T* sw = Tab + (size_t)NT * nm * nqp;                 // [nq] weights * |J|
  const size_t per_slot = (size_t)nb * (JVP ? 2 : 1) + (size_t)nq * M * D;
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
  T* sV = sW + nb;
  T* sF = sV + (JVP ? nb : 0);                          // [nq][M][D]
  const int bar = 1 + slot;
  for (int e = blockIdx.x * NSLOT + slot; e < E; e += gridDim.x * NSLOT) {
    for (int t = tid; t < nb; t += 256) {
      if (!Pv) sW[t] = W[(size_t)e * nb + t];
      if (JVP) sV[t] = V[(size_t)e * nb + t];
    }
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
    for (int q = tid; q < nq; q += 256) {
      S u[M], g[M][D];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        u[v] = T(0);
#pragma unroll
        for (int kk = 0; kk < D; ++kk) g[v][kk] = T(0);
      }
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
            T dp[D];
#pragma unroll
            for (int kk = 0; kk < D; ++kk) dp[kk] = tq[((size_t)(1 + kk) * nm + i) * nqp];
#pragma unroll
            for (int v = 0; v < M; ++v) {
              const T a = sV[v * nm + i];
              tv[v] += a * p;
#pragma unroll
              for (int kk = 0; kk < D; ++kk) th[v][kk] += a * dp[kk];
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
      for (int i = 0; interp && i < nm; ++i) {
        const T p = tq[(size_t)i * nqp];
        T dp[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) dp[kk] = tq[((size_t)(1 + kk) * nm + i) * nqp];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          S a;
          if constexpr (JVP) a = S(sW[v * nm + i], sV[v * nm + i]);
          else a = sW[v * nm + i];
          u[v] = u[v] + a * p;
#pragma unroll
          for (int kk = 0; kk < D; ++kk) g[v][kk] = g[v][kk] + a * dp[kk];
        }
      }
      if (!physical<D>(u, ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
      S F[M][D];
      flux_total<D, S, T>(u, g, F, ph);
      const T wq = sw[q];
      T* fo = sF + (size_t)q * M * D;
#pragma unroll
      for (int v = 0; v < M; ++v)
#pragma unroll
        for (int kk = 0; kk < D; ++kk) fo[v * D + kk] = wq * (JVP ? tan_part(F[v][kk]) : val(F[v][kk]));
    }
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
    for (int j = tid; j < nb; j += 256) {
      const int v = j / nm, i = j - v * nm;
      T acc[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) acc[kk] = T(0);
      const T* fv = sF + v * D;
      for (int q = 0; q < nq; ++q) {
#pragma unroll
        for (int kk = 0; kk < D; ++kk) acc[kk] += Tab[((size_t)(1 + kk) * nm + i) * nqp + q] * fv[(size_t)q * M * D + kk];
      }
      T a = T(0);
#pragma unroll
      for (int kk = 0; kk < D; ++kk) a -= acc[kk];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int em = mv.nbr[(e * D + k) * 2 + 0];
        a += slots[(((size_t)e * D + k) * 2 + 0) * nb + j];
        a += slots[(((size_t)em * D + k) * 2 + 1) * nb + j];
      }
      if (JVP) a += sigma * mv.detJ * sV[j];
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
  const size_t per_slot = (size_t)M.nb * (jvp ? 2 : 1) + (size_t)M.nq * M.m * M.d;
  const size_t n = (size_t)(1 + M.d) * M.nm * *nqp + M.nq;
  *bytes = n * sizeof(float) + 16 + VOL_SLOTS * ((per_slot + 3) / 4 * 4) * sizeof(float);
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return *bytes <= (size_t)smax;
}

template <class T>
static size_t face_smem(const Mesh& M, int fpc, bool jvp) {
  return sizeof(T) * (size_t)fpc *
         (2 * M.nb * (jvp ? 2 : 1) + 2 * M.nqf * M.m + M.nqf * M.m + 2 * M.nqf * M.m * M.d);
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
  int fpc = std::max(1, 128 / Ms.nqf);
  size_t fsm = face_smem<T>(Ms, fpc, JVP);
  while (fsm > 200 * 1024 && fpc > 1) fsm = face_smem<T>(Ms, --fpc, JVP);
  if (fsm > 48 * 1024)
    allow_max_smem(face_kernel<D, T, JVP>);
  int nfaces = D * Ms.E;
  if (parts & 1) {
    // 3-D: the face term by sum factorisation in FP64 (fewer of the FP64 pipe's
    // cycles: the residual 4.5 -> 3.8 ms at 16^3 p = 4) and in FP32 above 40
    // modes (at p = 4 the direct FP32 kernel is faster: 0.39 against 0.57 ms);
    // DG_NO_SUMFACT_FACE=1 keeps the direct kernel, DG_SUMFACT_FACE_MIN_MODES
    // moves the FP32 threshold (41 modes)
    const char* nsff = getenv("DG_NO_SUMFACT_FACE");
    const char* sfmin = getenv("DG_SUMFACT_FACE_MIN_MODES");
    const int min_modes = sfmin ? atoi(sfmin) : 41;
    cudaError_t e = cudaErrorNotSupported;
    if (D == 3 && !(nsff && nsff[0] == '1') && (std::is_same<T, double>::value || Ms.nm >= min_modes)) {
      e = launch_face_sf<T>(Ms, W, V, slots, JVP, JVP ? Pf : nullptr, st);
      if (e == cudaErrorNotSupported) (void)cudaGetLastError();
    }
    if (e == cudaErrorNotSupported) {
      note_launch();
      face_kernel<D, T, JVP><<<(nfaces + fpc - 1) / fpc, 128, fsm, st>>>(mv, ph, W, V, slots, Ms.status, fpc,
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
