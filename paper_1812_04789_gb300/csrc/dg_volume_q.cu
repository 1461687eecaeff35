// Volume term of the residual / exact JVP for the tensor-product space Q_p by
// sum factorisation (Sec. 3.1 eq. dg_ns, volume part; the paper's
// quadrilateral basis of Sec. 3).
//
// With phi_(a0,a1,a2)(xi) = L_a0(xi_0) L_a1(xi_1) L_a2(xi_2) and the tensor
// Gauss-Legendre points, the interpolation of u and of its d reference
// derivatives at all n_q = nq^d points is d successive one-dimensional
// contractions (the last one fused into the pointwise flux evaluation), and
// the projection  R_i -= sum_q w_q grad phi_i(q) . F(q)  is the transposed
// sequence: O((p+1) nq^d) work per contraction instead of O((p+1)^d nq^d).
// The total-degree space P_p is the subset a0 + a1 + a2 <= p of the same
// products, so its fields run through the same contractions with the other
// tensor coefficients zero (qidx = -1) and only its modes are written back.
// Interpolation (3-D): Z_s[v][a0][a1][q2] = sum_a2 W[v][a0 a1 a2] L^s_a2(q2)
// (s = value or derivative factor), Y_t[v][a0][q1][q2] = sum_a1 Z L^t_a1(q1)
// for the three patterns (L, L), (L', L)... needed by u, d/dxi_1, d/dxi_2,
// then per point u, du/dxi_0 from Y with L_a0, L'_a0.  Projection: P_j =
// sum_q0, Q_A, Q_B = sum_q1, R = sum_q2 with the matching factors; the
// metric 2/h_k multiplies each derivative factor.  One CTA per element;
// JVP: dual numbers carried as separate value / tangent arrays.
#include <algorithm>
#include <type_traits>

#include "dg_internal.h"

namespace dgk {

namespace {

struct QPlan {
  int n1, nq, nt, nqd;
  size_t oL, oW, oZ, oY, oF, oP, total;   // element offsets in shared memory (T)
};

__host__ __device__ constexpr size_t zmax(size_t a, size_t b) { return a > b ? a : b; }

// 3-D: two regions, each holding in turn what is live at that stage:
//   A: Z (interpolation), then F (pointwise fluxes), then R (modes)
//   B: the coefficients W, then Y (interpolation), then P, Q (projection)
// 2-D: W, the stages (Y, then P) and F apart.
template <int D>
__host__ __device__ inline QPlan q_plan(int p, int nq, int M, bool jvp) {
  QPlan P;
  P.n1 = p + 1;
  P.nq = nq;
  P.nt = 1;
  P.nqd = 1;
  for (int k = 0; k < D; ++k) {
    P.nt *= P.n1;
    P.nqd *= nq;
  }
  const size_t nc = jvp ? 2 : 1;   // value (+ tangent) copies
  const size_t n1 = P.n1;
  size_t o = 0;
  P.oL = o;
  o += 2 * n1 * nq + nq;
  if (D == 3) {
    const size_t nZ = 2 * M * n1 * n1 * nq, nY = 3 * M * n1 * nq * nq;
    const size_t nP = M * n1 * nq * nq, nQ = M * n1 * n1 * nq;
    const size_t A = zmax(nc * nZ, (size_t)D * M * P.nqd);
    const size_t B = zmax(zmax(nc * M * P.nt, nc * nY), 3 * nP + 2 * nQ);
    P.oZ = P.oF = o;
    o += A;
    P.oW = P.oY = P.oP = o;
    o += B;
  } else {
    P.oW = o;
    o += nc * M * P.nt;
    P.oY = P.oP = P.oZ = o;
    o += zmax(nc * 2 * M * n1 * nq, (size_t)2 * M * n1 * nq);
    P.oF = o;
    o += (size_t)D * M * P.nqd;
  }
  P.total = o;
  return P;
}

template <int D, class T, bool JVP>
__global__ void __launch_bounds__(256) volume_q_kernel(MeshView<T> mv, Phys<T> ph, const T* __restrict__ l1g,
                                                       const int* __restrict__ qidx, const T* __restrict__ W,
                                                       const T* __restrict__ V, const T* __restrict__ slots,
                                                       const T* __restrict__ Src, T sigma, T* __restrict__ out,
                                                       int* status, int p, int nq, T m0, T m1, T m2) {
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  constexpr int M = D + 2, NC = JVP ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const QPlan P = q_plan<D>(p, nq, M, JVP);
  const int n1 = P.n1, nt = P.nt, nqd = P.nqd, nb = mv.nb, E = mv.E;
  const T* L = sm + P.oL;            // L[a][q]
  const T* dL = L + n1 * nq;         // dL[a][q]
  const T* w1 = dL + n1 * nq;        // w[q]
  T* Wt = sm + P.oW;                 // [c][v][t], c = value, tangent
  T* F = sm + P.oF;                  // [k][v][q]: w_q |J| F (value or tangent)
  const T met[3] = {m0, m1, m2};
  for (int t = threadIdx.x; t < 2 * n1 * nq + nq; t += blockDim.x) sm[P.oL + t] = l1g[t];
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    for (int t = threadIdx.x; t < M * nt; t += blockDim.x) {
      const int v = t / nt, ti = t - v * nt, i = qidx[ti];
      Wt[t] = i >= 0 ? W[(size_t)e * nb + v * mv.nm + i] : T(0);
      if (JVP) Wt[M * nt + t] = i >= 0 ? V[(size_t)e * nb + v * mv.nm + i] : T(0);
    }
    __syncthreads();
    // ---------------- interpolation
    if (D == 3) {
      const int nZ = 2 * M * n1 * n1 * nq, nY = 3 * M * n1 * nq * nq;
      T* Z = sm + P.oZ;       // [c][s][v][a0][a1][q2]
      T* Y = sm + P.oY;       // [c][t][v][a0][q1][q2] (over W: Z is complete)
      for (int t = threadIdx.x; t < NC * nZ; t += blockDim.x) {
        const int c = t / nZ, r = t - c * nZ;
        const int q2 = r % nq, a1 = (r / nq) % n1, a0 = (r / (nq * n1)) % n1, v = (r / (nq * n1 * n1)) % M,
                  s = r / (nq * n1 * n1 * M);
        const T* Ls = s ? dL : L;
        const T* w = Wt + (size_t)c * M * nt + v * nt + a0 + n1 * a1;
        T acc = T(0);
        for (int a2 = 0; a2 < n1; ++a2) acc += w[n1 * n1 * a2] * Ls[a2 * nq + q2];
        Z[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < NC * nY; t += blockDim.x) {
        const int c = t / nY, r = t - c * nY;
        const int q2 = r % nq, q1 = (r / nq) % nq, a0 = (r / (nq * nq)) % n1, v = (r / (nq * nq * n1)) % M,
                  ts = r / (nq * nq * n1 * M);
        // ts 0: (L on a1, L on a2); 1: (L' on a1, L on a2); 2: (L on a1, L' on a2)
        const T* Lt = ts == 1 ? dL : L;
        const T* z = Z + (size_t)c * nZ + (((size_t)(ts == 2 ? 1 : 0) * M + v) * n1 + a0) * n1 * nq + q2;
        T acc = T(0);
        for (int a1 = 0; a1 < n1; ++a1) acc += z[a1 * nq] * Lt[a1 * nq + q1];
        Y[t] = acc;
      }
    } else {
      const int nY = 2 * M * n1 * nq;
      T* Y = sm + P.oY;   // [c][s][v][a0][q1]
      for (int t = threadIdx.x; t < NC * nY; t += blockDim.x) {
        const int c = t / nY, r = t - c * nY;
        const int q1 = r % nq, a0 = (r / nq) % n1, v = (r / (nq * n1)) % M, s = r / (nq * n1 * M);
        const T* Ls = s ? dL : L;
        const T* w = Wt + (size_t)c * M * nt + v * nt + a0;
        T acc = T(0);
        for (int a1 = 0; a1 < n1; ++a1) acc += w[n1 * a1] * Ls[a1 * nq + q1];
        Y[t] = acc;
      }
    }
    __syncthreads();
    // ---------------- pointwise flux (the last contraction fused in)
    for (int q = threadIdx.x; q < nqd; q += blockDim.x) {
      const int q0 = q % nq, qr = q / nq;   // qr = q1 (2-D) or q1 + nq q2 (3-D)
      const int yq = D == 3 ? (qr % nq) * nq + qr / nq : qr;   // (q1, q2) in the Y layout, q2 fastest
      S u[M], g[M][D];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        T uu[NC], gg[NC][D];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          uu[c] = T(0);
#pragma unroll
          for (int k = 0; k < D; ++k) gg[c][k] = T(0);
        }
        if (D == 3) {
          const int nY = 3 * M * n1 * nq * nq;
          const T* Y = sm + P.oY;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const T* y0 = Y + (size_t)c * nY + ((size_t)(0 * M + v) * n1) * nq * nq + yq;
            const T* y1 = Y + (size_t)c * nY + ((size_t)(1 * M + v) * n1) * nq * nq + yq;
            const T* y2 = Y + (size_t)c * nY + ((size_t)(2 * M + v) * n1) * nq * nq + yq;
            for (int a0 = 0; a0 < n1; ++a0) {
              const T la = L[a0 * nq + q0], da = dL[a0 * nq + q0];
              const T v0 = y0[a0 * nq * nq];
              uu[c] += v0 * la;
              gg[c][0] += v0 * da;
              gg[c][1] += y1[a0 * nq * nq] * la;
              gg[c][2 % D] += y2[a0 * nq * nq] * la;
            }
          }
        } else {
          const int nY = 2 * M * n1 * nq;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const T* y0 = sm + P.oY + (size_t)c * nY + ((size_t)(0 * M + v) * n1) * nq + yq;
            const T* y1 = sm + P.oY + (size_t)c * nY + ((size_t)(1 * M + v) * n1) * nq + yq;
            for (int a0 = 0; a0 < n1; ++a0) {
              const T la = L[a0 * nq + q0], da = dL[a0 * nq + q0];
              const T v0 = y0[a0 * nq];
              uu[c] += v0 * la;
              gg[c][0] += v0 * da;
              gg[c][1] += y1[a0 * nq] * la;
            }
          }
        }
        if constexpr (JVP) {
          u[v] = S(uu[0], uu[1]);
#pragma unroll
          for (int k = 0; k < D; ++k) g[v][k] = S(gg[0][k] * met[k], gg[1][k] * met[k]);
        } else {
          u[v] = uu[0];
#pragma unroll
          for (int k = 0; k < D; ++k) g[v][k] = gg[0][k] * met[k];
        }
      }
      if (!physical<D>(u, ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
      S Fl[M][D];
      flux_total<D, S, T>(u, g, Fl, ph);
      T wq = mv.detJ * w1[q0];
      int r = qr;
#pragma unroll
      for (int k = 1; k < D; ++k) {
        wq *= w1[r % nq];
        r /= nq;
      }
#pragma unroll
      for (int v = 0; v < M; ++v)
#pragma unroll
        for (int k = 0; k < D; ++k) F[((size_t)k * M + v) * nqd + q] = wq * (JVP ? tan_part(Fl[v][k]) : val(Fl[v][k]));
    }
    __syncthreads();
    // ---------------- projection onto grad phi
    T* R = nullptr;   // [v][t] in the last stage's buffer
    if (D == 3) {
      const int nP = M * n1 * nq * nq, nQ = M * n1 * n1 * nq;
      T* Pb = sm + P.oP;      // [j][v][a0][q1][q2] (over Y: F is complete)
      T* Qb = Pb + 3 * nP;    // [A, B][v][a0][a1][q2]
      for (int t = threadIdx.x; t < 3 * nP; t += blockDim.x) {
        const int j = t / nP, r = t - j * nP;
        const int q12 = r % (nq * nq), a0 = (r / (nq * nq)) % n1, v = r / (nq * nq * n1);
        const T* f = F + ((size_t)j * M + v) * nqd + (size_t)q12 * nq;
        const T* La = (j == 0 ? dL : L) + a0 * nq;
        T acc = T(0);
        for (int q0 = 0; q0 < nq; ++q0) acc += La[q0] * f[q0];
        Pb[t] = j == 0 ? acc * met[0] : acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 2 * nQ; t += blockDim.x) {
        const int j = t / nQ, r = t - j * nQ;
        const int q2 = r % nq, a1 = (r / nq) % n1, a0 = (r / (nq * n1)) % n1, v = r / (nq * n1 * n1);
        T acc = T(0);
        if (j == 0) {
          const T* p0 = Pb + (((size_t)0 * M + v) * n1 + a0) * nq * nq + (size_t)q2 * nq;
          const T* p1 = Pb + (((size_t)1 * M + v) * n1 + a0) * nq * nq + (size_t)q2 * nq;
          for (int q1 = 0; q1 < nq; ++q1)
            acc += L[a1 * nq + q1] * p0[q1] + dL[a1 * nq + q1] * met[1] * p1[q1];
        } else {
          const T* p2 = Pb + (((size_t)2 * M + v) * n1 + a0) * nq * nq + (size_t)q2 * nq;
          for (int q1 = 0; q1 < nq; ++q1) acc += L[a1 * nq + q1] * p2[q1];
        }
        Qb[t] = acc;
      }
      __syncthreads();
      R = F;   // F is dead: reuse it for R[v][t]
      for (int t = threadIdx.x; t < M * nt; t += blockDim.x) {
        const int v = t / nt, ti = t - v * nt;
        const int a0 = ti % n1, a1 = (ti / n1) % n1, a2 = ti / (n1 * n1);
        const T* qa = Qb + (((size_t)0 * M + v) * n1 + a0) * n1 * nq + (size_t)a1 * nq;
        const T* qb = Qb + (((size_t)1 * M + v) * n1 + a0) * n1 * nq + (size_t)a1 * nq;
        T acc = T(0);
        for (int q2 = 0; q2 < nq; ++q2) acc += L[a2 * nq + q2] * qa[q2] + dL[a2 * nq + q2] * met[2 % D] * qb[q2];
        R[t] = -acc;
      }
    } else {
      const int nP = M * n1 * nq;
      T* Pb = sm + P.oP;   // [j][v][a0][q1]
      for (int t = threadIdx.x; t < 2 * nP; t += blockDim.x) {
        const int j = t / nP, r = t - j * nP;
        const int q1 = r % nq, a0 = (r / nq) % n1, v = r / (nq * n1);
        const T* f = F + ((size_t)j * M + v) * nqd + (size_t)q1 * nq;
        const T* La = (j == 0 ? dL : L) + a0 * nq;
        T acc = T(0);
        for (int q0 = 0; q0 < nq; ++q0) acc += La[q0] * f[q0];
        Pb[t] = j == 0 ? acc * met[0] : acc;
      }
      __syncthreads();
      R = F;
      for (int t = threadIdx.x; t < M * nt; t += blockDim.x) {
        const int v = t / nt, ti = t - v * nt;
        const int a0 = ti % n1, a1 = ti / n1;
        const T* p0 = Pb + ((size_t)0 * M + v) * n1 * nq + (size_t)a0 * nq;
        const T* p1 = Pb + ((size_t)1 * M + v) * n1 * nq + (size_t)a0 * nq;
        T acc = T(0);
        for (int q1 = 0; q1 < nq; ++q1) acc += L[a1 * nq + q1] * p0[q1] + dL[a1 * nq + q1] * met[1] * p1[q1];
        R[t] = -acc;
      }
    }
    __syncthreads();
    // ---------------- modes: volume part + face slots (fixed order) + sigma |J| v or - source
    for (int t = threadIdx.x; t < M * nt; t += blockDim.x) {
      const int v = t / nt, ti = t - v * nt, i = qidx[ti], j = v * mv.nm + i;
      if (i < 0) continue;   // a tensor coefficient outside P_p
      T acc = R[t];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int em = mv.nbr[(e * D + k) * 2 + 0];
        acc += slots[(((size_t)e * D + k) * 2 + 0) * nb + j];
        acc += slots[(((size_t)em * D + k) * 2 + 1) * nb + j];
      }
      if (JVP) acc += sigma * mv.detJ * V[(size_t)e * nb + j];
      else if (Src) acc -= Src[(size_t)e * nb + j];
      out[(size_t)e * nb + j] = acc;
    }
    __syncthreads();
  }
}

template <int D, class T, bool JVP>
cudaError_t run_q(const Mesh& Ms, const T* W, const T* V, const T* S, T sigma, T* out, cudaStream_t st) {
  const QPlan P = q_plan<D>(Ms.p, Ms.nq1d, Ms.m, JVP);
  const size_t smem = P.total * sizeof(T);
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)smax) return cudaErrorNotSupported;
  cudaError_t e = allow_max_smem(volume_q_kernel<D, T, JVP>);
  if (e != cudaSuccess) return e;
  const T* l1 = std::is_same<T, double>::value ? (const T*)Ms.t64.l1d : (const T*)Ms.t32.l1d;
  const T* slots = std::is_same<T, double>::value ? (const T*)Ms.t64.slots : (const T*)Ms.t32.slots;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, volume_q_kernel<D, T, JVP>, 256, smem);
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(Ms.E, std::max(1, occ) * nsm);
  const T m0 = (T)(2.0 / Ms.h[0]), m1 = (T)(2.0 / Ms.h[1]), m2 = (T)(D == 3 ? 2.0 / Ms.h[2] : 0.0);
  note_launch();
  volume_q_kernel<D, T, JVP><<<grid, 256, smem, st>>>(Ms.view<T>(), Ms.phys_t<T>(), l1, Ms.qidx, W, V, slots, S,
                                                      sigma, out, Ms.status, Ms.p, Ms.nq1d, m0, m1, m2);
  return cudaGetLastError();
}

}  // namespace

template <class T>
cudaError_t launch_volume_q(const Mesh& M, const T* W, const T* V, const T* S, T sigma, bool jvp, T* out,
                            cudaStream_t st) {
  if (M.kind != DG_MESH_STRUCTURED || !M.qidx) return cudaErrorNotSupported;
  if (M.d == 2)
    return jvp ? run_q<2, T, true>(M, W, V, S, sigma, out, st) : run_q<2, T, false>(M, W, V, S, sigma, out, st);
  return jvp ? run_q<3, T, true>(M, W, V, S, sigma, out, st) : run_q<3, T, false>(M, W, V, S, sigma, out, st);
}
template cudaError_t launch_volume_q<double>(const Mesh&, const double*, const double*, const double*, double,
                                             bool, double*, cudaStream_t);
template cudaError_t launch_volume_q<float>(const Mesh&, const float*, const float*, const float*, float, bool,
                                            float*, cudaStream_t);

}  // namespace dgk
