// Pieces shared by the two block-probing kernels (dg_blocks.cu: SIMT, every
// precision; dg_probe_tc.cu: tensor cores, FP32): the tangent of the face-point
// outputs for a unit seed, and the per-element staging of W with the primal
// traces at the volume and face quadrature points (Sec. 3.1).
#pragma once
#include "dg_internal.h"

namespace dgk {

// Tangent of the face-point outputs for a unit seed: so/sgo on the own trace,
// sn/sgn on the neighbour's.  Outputs: numerical flux fp[v], lifting integrands
// GL[v], GR[v] of the face's +k / -k sides, and the element's own dual tensor.
template <int D, class T>
__device__ __forceinline__ void face_point_tangent(const T* pu_own, const T* pu_nb, int k, int side,
                                                   int w, T so, const T* sgo, T sn, const T* sgn,
                                                   const Phys<T>& ph, T* bGL, T* bGR, T* bFp,
                                                   T* bDo) {
  using S = Dual<T>;
  constexpr int M = D + 2;
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

// Stage W of element e and its 2d neighbours into cW (face order s = 2k + side)
// and evaluate the primal traces: cU[q] = (u, grad u) at the volume points
// (when with_volume) and cFU[(s, side, q)] on both sides of every face.
// Flags a non-physical state in *status.  Contains two block barriers.
template <int D, class T>
__device__ __forceinline__ void probe_stage_primal(const MeshView<T>& mv, const Phys<T>& ph,
                                                   const T* __restrict__ W, int e, const int* nbrs, T* cW,
                                                   T* cU, T* cFU, bool with_volume, int* status) {
  constexpr int M = D + 2, NF = 2 * D, PU = M * (1 + D);
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, nqf = mv.nqf;
  // ---- stage W of the element and its neighbours (face order s = 2k + side)
  for (int t = threadIdx.x; t < (1 + NF) * nb; t += blockDim.x) {
    int who = t / nb, j = t % nb;
    int el = who == 0 ? e : nbrs[who - 1];
    cW[t] = W[(size_t)el * nb + j];
  }
  __syncthreads();
  // ---- primal traces: volume points and both sides of every face
  for (int t = (with_volume ? 0 : nq) + (int)threadIdx.x; t < nq + NF * 2 * nqf; t += blockDim.x) {
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
    if (!physical<D>(u, ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
#pragma unroll
    for (int v = 0; v < M; ++v) {
      dst[v] = u[v];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) dst[M + v * D + kk] = g[v][kk];
    }
  }
  __syncthreads();
}

}  // namespace dgk
