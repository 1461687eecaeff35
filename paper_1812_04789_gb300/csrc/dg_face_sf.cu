// Face term of the residual / exact JVP on 3-D meshes by sum factorisation
// (Sec. 3.1 eq. dg_ns face terms, eq. visc_flux and the lifting of eq. re).
//
// On the face k of an element the basis functions are products
// L_a(xi_k = +-1) L_b(xi_t0) L_c(xi_t1) (t0 < t1 the two other directions) and
// the face points a tensor grid (b0, b1) of the same Gauss-Legendre points,
// q = b0 + nq b1.  The traces of a field and of its gradient at all n_qf points
// are then three short contractions instead of one over all modes:
//   S1  c0[a0][a1] = sum_ak w L_ak(+-1),  c1[a0][a1] = sum_ak w L'_ak(+-1)
//   S2  d0[a0][b1] = sum_a1 c0 L_a1(b1),  d1 = sum_a1 c0 L'_a1(b1),  d2 = sum_a1 c1 L_a1(b1)
//   per point: u = sum_a0 d0 L_a0(b0), du/dt0 = sum d0 L'_a0(b0), du/dt1 = sum d1 L_a0(b0),
//              du/dn = sum d2 L_a0(b0)   (each derivative times its metric 2/h)
// and the projection of the face fluxes onto both elements' test functions is
// the transposed sequence (X over b0, Y over b1, then the end values).  The
// total-degree space P_p is the subset a_k + a0 + a1 <= p of these products
// (qidx maps a tensor index to its mode, -1 outside P_p), Q_p all of them.
// Pointwise physics and the BR2 lifting are those of face_kernel
// (csrc/dg_residual.cu), point for point.
#include <algorithm>
#include <type_traits>

#include "dg_internal.h"

namespace dgk {

namespace {

// shared-memory plan (elements of T); NC = interpolated real fields per side
struct FsfPlan {
  int n1, nq, nqf, NC;
  size_t oW, oV, oG, oF, oD, oS, oT, per_face, total;
};

__host__ __device__ inline FsfPlan fsf_plan(int p, int nq, int nb, int M, bool jvp, bool cached, int fpc) {
  FsfPlan P;
  P.n1 = p + 1;
  P.nq = nq;
  P.nqf = nq * nq;
  const bool haveW = !(jvp && cached);
  P.NC = (haveW ? 1 : 0) + (jvp ? 1 : 0);
  // the coefficients (read by S1 only) share their space with the point values
  // (written from phase 1 on, after S2)
  P.oW = 0;
  P.oV = haveW ? (size_t)fpc * 2 * nb : 0;
  const size_t coef = P.oV + (jvp ? (size_t)fpc * 2 * nb : 0);
  P.oG = 0;
  P.oF = (size_t)fpc * 2 * P.nqf * M;
  P.oD = P.oF + (size_t)fpc * P.nqf * M;
  const size_t pts = P.oD + (size_t)fpc * 2 * P.nqf * M * 3;
  size_t o = coef > pts ? coef : pts;
  const size_t interp = (size_t)2 * P.NC * M * (2 * P.n1 * P.n1 + 3 * P.n1 * nq);
  const size_t proj = (size_t)2 * M * (3 * P.n1 * nq + 2 * P.n1 * P.n1);
  P.per_face = interp > proj ? interp : proj;
  P.oS = o;
  o += (size_t)fpc * P.per_face;
  P.oT = o;                                            // L[n1][nq] dL[n1][nq] Le[2][n1] dLe[2][n1]
  o += (size_t)2 * P.n1 * nq + 4 * P.n1;
  P.total = o;
  return P;
}

// component d of a triple held in scalars (no run-time indexing of local arrays)
template <class T>
__device__ __forceinline__ T pick3(int d, T x0, T x1, T x2) {
  return d == 0 ? x0 : (d == 1 ? x1 : x2);
}

}  // namespace

template <class T, bool JVP>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2)
    face_sf_kernel(MeshView<T> mv, Phys<T> ph, const T* __restrict__ W, const T* __restrict__ V,
                   T* __restrict__ slots, int* status, int fpc, const T* __restrict__ Pf, const T* __restrict__ l1g,
                   const int* __restrict__ qidx, int p, int nq, T m0, T m1, T m2) {
  using S = typename std::conditional<JVP, Dual<T>, T>::type;
  constexpr int D = 3, M = D + 2, PU = M * (1 + D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int nb = mv.nb, nm = mv.nm, nqf = mv.nqf, E = mv.E;
  const bool cached = JVP && Pf != nullptr;
  const FsfPlan P = fsf_plan(p, nq, nb, M, JVP, cached, fpc);
  const int n1 = P.n1, NC = P.NC;
  const bool haveW = !cached;
  const int nfaces = D * E, f0 = blockIdx.x * fpc, nloc = min(fpc, nfaces - f0);
  if (nloc <= 0) return;
  T* sW = sm + P.oW;               // [fpc][2][nb]  state (not with cached traces), until S1
  T* sV = sm + P.oV;               // [fpc][2][nb]  direction (JVP), until S1
  T* sG = sm + P.oG;               // [fpc][2][nqf][M]
  T* sF = sm + P.oF;               // [fpc][nqf][M]
  T* sD = sm + P.oD;               // [fpc][2][nqf][M][D]
  T* sS = sm + P.oS;               // [fpc][per_face]: contraction stages
  T* tab = sm + P.oT;
  const T* L = tab;                // L[a][b]
  const T* dL = tab + n1 * nq;     // dL[a][b] (reference derivative)
  const T* Le = dL + n1 * nq;      // Le[end][a], end 0 at -1, 1 at +1
  const T* dLe = Le + 2 * n1;
  for (int t = threadIdx.x; t < 2 * n1 * nq; t += blockDim.x) tab[t] = l1g[t];
  for (int t = threadIdx.x; t < 4 * n1; t += blockDim.x) tab[2 * n1 * nq + t] = l1g[2 * n1 * nq + nq + t];
  // phase 0: the modal coefficients of both elements of every face
  for (int t = threadIdx.x; t < nloc * 2 * nb; t += blockDim.x) {
    const int fl = t / (2 * nb), r = t % (2 * nb), side = r / nb, j = r % nb;
    const int f = f0 + fl, k = f / E, e = f % E;
    const int el = side == 0 ? e : mv.nbr[(e * D + k) * 2 + 1];
    if (haveW) sW[t] = W[(size_t)el * nb + j];
    if (JVP) sV[t] = V[(size_t)el * nb + j];
  }
  __syncthreads();
  // S1: collapse the normal direction with the end values (L and L')
  const int n1s = n1 * n1, s1sz = 2 * NC * M * 2 * n1s;
  for (int t = threadIdx.x; t < nloc * s1sz; t += blockDim.x) {
    const int fl = t / s1sz;
    int r = t - fl * s1sz;
    const int a1 = r % n1;
    r /= n1;
    const int a0 = r % n1;
    r /= n1;
    const int w2 = r % 2;
    r /= 2;
    const int v = r % M;
    r /= M;
    const int c = r % NC, side = r / NC;
    const int k = (f0 + fl) / E, t0 = k == 0 ? 1 : 0, t1 = k == 2 ? 1 : 2;
    const int end = side == 0 ? 1 : 0;       // the element on side 0 meets the face at xi_k = +1
    const T* Ev = (w2 ? dLe : Le) + end * n1;
    const T* fld = ((haveW && c == 0) ? sW : sV) + ((size_t)fl * 2 + side) * nb + v * nm;
    T acc = T(0);
    const int sk = pick3(k, 1, n1, n1s), base = a0 * pick3(t0, 1, n1, n1s) + a1 * pick3(t1, 1, n1, n1s);
    for (int ak = 0; ak < n1; ++ak) {
      const int i = qidx[base + ak * sk];
      if (i >= 0) acc += fld[i] * Ev[ak];
    }
    sS[(size_t)fl * P.per_face + (t - fl * s1sz)] = acc;
  }
  __syncthreads();
  // S2: contract the second tangential direction: d0 = c0 L, d1 = c0 L', d2 = c1 L
  const int s2sz = 2 * NC * M * 3 * n1 * nq;
  for (int t = threadIdx.x; t < nloc * s2sz; t += blockDim.x) {
    const int fl = t / s2sz;
    int r = t - fl * s2sz;
    const int b1 = r % nq;
    r /= nq;
    const int a0 = r % n1;
    r /= n1;
    const int ty = r % 3;
    r /= 3;
    const int scv = r;                       // (side, c, v)
    const T* s1 = sS + (size_t)fl * P.per_face + ((size_t)scv * 2 + (ty == 2 ? 1 : 0)) * n1s + a0 * n1;
    const T* Lt = ty == 1 ? dL : L;
    T acc = T(0);
    for (int a1 = 0; a1 < n1; ++a1) acc += s1[a1] * Lt[a1 * nq + b1];
    sS[(size_t)fl * P.per_face + s1sz + (t - fl * s2sz)] = acc;
  }
  __syncthreads();
  // phase 1: traces at the face points from the S2 stage, pointwise physics
  // (as face_kernel: with cached traces a JVP takes the state's from the cache)
  for (int t = threadIdx.x; t < nloc * nqf; t += blockDim.x) {
    const int fl = t / nqf, q = t % nqf, b0 = q % nq, b1 = q / nq;
    const int f = f0 + fl, k = f / E, t0 = k == 0 ? 1 : 0, t1 = k == 2 ? 1 : 2;
    const T* s2 = sS + (size_t)fl * P.per_face + s1sz;
    S uS[2][M], gS[2][M][D];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        T val[2] = {T(0), T(0)}, gn[2] = {T(0), T(0)}, g0[2] = {T(0), T(0)}, g1[2] = {T(0), T(0)};
        for (int c = 0; c < NC; ++c) {
          const T* d = s2 + ((size_t)((side * NC + c) * M + v) * 3) * n1 * nq + b1;   // [ty][a0][b1]
          T u_ = T(0), ut0 = T(0), ut1 = T(0), un = T(0);
          for (int a0 = 0; a0 < n1; ++a0) {
            const T la = L[a0 * nq + b0], da = dL[a0 * nq + b0];
            const T d0 = d[(size_t)a0 * nq], d1 = d[(size_t)(n1 + a0) * nq], d2 = d[(size_t)(2 * n1 + a0) * nq];
            u_ += d0 * la;
            ut0 += d0 * da;
            ut1 += d1 * la;
            un += d2 * la;
          }
          val[c] = u_;
          gn[c] = un * pick3(k, m0, m1, m2);
          g0[c] = ut0 * pick3(t0, m0, m1, m2);
          g1[c] = ut1 * pick3(t1, m0, m1, m2);
        }
        // the gradient component of physical direction kk: normal, first or second tangential
#define GCOMP(c, kk) ((kk) == k ? gn[c] : ((kk) == t0 ? g0[c] : g1[c]))
        if constexpr (JVP) {
          if (cached) {
            const T* cc = Pf + ((size_t)(f0 + fl) * nqf + q) * 2 * PU + side * PU;
            uS[side][v] = S(cc[v], val[0]);
#pragma unroll
            for (int kk = 0; kk < D; ++kk) gS[side][v][kk] = S(cc[M + v * D + kk], GCOMP(0, kk));
          } else {
            uS[side][v] = S(val[0], val[1]);
#pragma unroll
            for (int kk = 0; kk < D; ++kk) gS[side][v][kk] = S(GCOMP(0, kk), GCOMP(1, kk));
          }
        } else {
          uS[side][v] = val[0];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) gS[side][v][kk] = GCOMP(0, kk);
        }
#undef GCOMP
      }
    }
    if (!physical<D>(uS[0], ph.gm1) || !physical<D>(uS[1], ph.gm1)) atomicOr(status, ST_NONPHYSICAL);
    S fp[M], GLn[M], GRn[M], DL[M][D], DR[M][D];
    face_point_k<D, S, T>(k, uS[0], gS[0], uS[1], gS[1], ph, fp, GLn, GRn, DL, DR);
    T* gq0 = sG + ((size_t)fl * 2 * nqf + q) * M;
    T* gq1 = sG + ((size_t)(fl * 2 + 1) * nqf + q) * M;
    T* fo = sF + ((size_t)fl * nqf + q) * M;
    T* dq0 = sD + (((size_t)fl * 2) * nqf + q) * M * D;
    T* dq1 = sD + (((size_t)fl * 2 + 1) * nqf + q) * M * D;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      fo[v] = JVP ? tan_part(fp[v]) : val(fp[v]);
      gq0[v] = JVP ? tan_part(GLn[v]) : val(GLn[v]);
      gq1[v] = JVP ? tan_part(GRn[v]) : val(GRn[v]);
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        dq0[v * D + kk] = JVP ? tan_part(DL[v][kk]) : val(DL[v][kk]);
        dq1[v * D + kk] = JVP ? tan_part(DR[v][kk]) : val(DR[v][kk]);
      }
    }
  }
  __syncthreads();
  // phase 2: BR2 lifting on both sides, fhat = Roe + {F_v}.n + eta {delta}.n (as face_kernel)
  for (int t = threadIdx.x; t < nloc * nqf; t += blockDim.x) {
    const int fl = t / nqf, q = t % nqf;
    const int k = (f0 + fl) / E;
    const T* PL = mv.lift + (size_t)(2 * k + 1) * nqf * nqf + q;   // column q2 at PL[q2 * nqf]
    const T* PR = mv.lift + (size_t)(2 * k) * nqf * nqf + q;
    T dl[M], dr[M];
#pragma unroll
    for (int v = 0; v < M; ++v) dl[v] = dr[v] = T(0);
    for (int q2 = 0; q2 < nqf; ++q2) {
      const T a = PL[(size_t)q2 * nqf], b = PR[(size_t)q2 * nqf];
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
  // phase 3: projection onto both elements' test functions by the transposed
  // contractions.  Per side and variable, with the point values
  //   A = sgn fw Fo,  P = -fw Dd_t0 m_t0,  Q = -fw Dd_t1 m_t1,  N = -fw Dd_n m_n:
  //   X: XA[a0][b1] = sum_b0 A L_a0(b0) + P L'_a0(b0),  XQ = sum_b0 Q L_a0(b0),  XN = sum_b0 N L_a0(b0)
  //   Y: YA[a0][a1] = sum_b1 XA L_a1(b1) + XQ L'_a1(b1),  YN = sum_b1 XN L_a1(b1)
  //   slot(mode (ak, a0, a1)) = L_ak(+-1) YA + L'_ak(+-1) YN
  const int xsz = 2 * M * 3 * n1 * nq;
  for (int t = threadIdx.x; t < nloc * xsz; t += blockDim.x) {
    const int fl = t / xsz;
    int r = t - fl * xsz;
    const int b1 = r % nq;
    r /= nq;
    const int a0 = r % n1;
    r /= n1;
    const int kind = r % 3;
    r /= 3;
    const int v = r % M, side = r / M;
    const int k = (f0 + fl) / E, t0 = k == 0 ? 1 : 0, t1 = k == 2 ? 1 : 2;
    const T sgn = side == 0 ? T(1) : T(-1);
    const T mk = pick3(k, m0, m1, m2), mt0 = pick3(t0, m0, m1, m2), mt1 = pick3(t1, m0, m1, m2);
    const T* fw = mv.fw + (size_t)k * nqf;
    const T* Fo = sF + (size_t)fl * nqf * M;
    const T* Dd = sD + ((size_t)(fl * 2 + side) * nqf) * M * D;
    T acc = T(0);
    for (int b0 = 0; b0 < nq; ++b0) {
      const int q = b0 + nq * b1;
      const T la = L[a0 * nq + b0];
      const T* dd = Dd + ((size_t)q * M + v) * D;
      if (kind == 0)
        acc += fw[q] * (sgn * Fo[q * M + v] * la - dd[t0] * mt0 * dL[a0 * nq + b0]);
      else if (kind == 1)
        acc -= fw[q] * dd[t1] * mt1 * la;
      else
        acc -= fw[q] * dd[k] * mk * la;
    }
    sS[(size_t)fl * P.per_face + (t - fl * xsz)] = acc;
  }
  __syncthreads();
  const int ysz = 2 * M * 2 * n1s;
  for (int t = threadIdx.x; t < nloc * ysz; t += blockDim.x) {
    const int fl = t / ysz;
    int r = t - fl * ysz;
    const int a1 = r % n1;
    r /= n1;
    const int a0 = r % n1;
    r /= n1;
    const int kind = r % 2;
    const int sv = r / 2;                    // (side, v)
    const T* X = sS + (size_t)fl * P.per_face + (size_t)sv * 3 * n1 * nq + a0 * nq;   // [kind][a0][b1]
    T acc = T(0);
    if (kind == 0) {
      for (int b1 = 0; b1 < nq; ++b1) acc += X[b1] * L[a1 * nq + b1] + X[(size_t)n1 * nq + b1] * dL[a1 * nq + b1];
    } else {
      for (int b1 = 0; b1 < nq; ++b1) acc += X[(size_t)2 * n1 * nq + b1] * L[a1 * nq + b1];
    }
    sS[(size_t)fl * P.per_face + xsz + (t - fl * ysz)] = acc;
  }
  __syncthreads();
  const int n13 = n1s * n1, osz = 2 * M * n13;
  for (int t = threadIdx.x; t < nloc * osz; t += blockDim.x) {
    const int fl = t / osz;
    int r = t - fl * osz;
    const int tt = r % n13;
    r /= n13;
    const int v = r % M, side = r / M;
    const int i = qidx[tt];
    if (i < 0) continue;                     // a tensor product outside P_p
    const int f = f0 + fl, k = f / E, e = f % E, t0 = k == 0 ? 1 : 0, t1 = k == 2 ? 1 : 2;
    const int x0 = tt % n1, x1 = (tt / n1) % n1, x2 = tt / n1s;
    const int ak = pick3(k, x0, x1, x2), a0 = pick3(t0, x0, x1, x2), a1 = pick3(t1, x0, x1, x2);
    const int end = side == 0 ? 1 : 0;
    const T* Y = sS + (size_t)fl * P.per_face + xsz + (size_t)(side * M + v) * 2 * n1s + a0 * n1 + a1;
    slots[(((size_t)e * D + k) * 2 + side) * nb + v * nm + i] = Le[end * n1 + ak] * Y[0] + dLe[end * n1 + ak] * Y[n1s];
  }
}

template <class T, bool JVP>
static cudaError_t run_face_sf(const Mesh& Ms, const T* W, const T* V, T* slots, const T* Pf, cudaStream_t st) {
  const bool cached = JVP && Pf != nullptr;
  int fpc = std::max(1, 128 / Ms.nqf);
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  size_t smem = fsf_plan(Ms.p, Ms.nq1d, Ms.nb, Ms.m, JVP, cached, fpc).total * sizeof(T);
  while (smem > (size_t)smax - 1024 && fpc > 1) smem = fsf_plan(Ms.p, Ms.nq1d, Ms.nb, Ms.m, JVP, cached, --fpc).total * sizeof(T);
  if (smem > (size_t)smax - 1024) return cudaErrorNotSupported;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(face_sf_kernel<T, JVP>);
    if (e != cudaSuccess) return e;
  }
  const T* l1 = std::is_same<T, double>::value ? (const T*)Ms.t64.l1d : (const T*)Ms.t32.l1d;
  const T m0 = (T)(2.0 / Ms.h[0]), m1 = (T)(2.0 / Ms.h[1]), m2 = (T)(2.0 / Ms.h[2]);
  const int nfaces = 3 * Ms.E;
  note_launch();
  face_sf_kernel<T, JVP><<<(nfaces + fpc - 1) / fpc, 128, smem, st>>>(Ms.view<T>(), Ms.phys_t<T>(), W, V, slots,
                                                                     Ms.status, fpc, cached ? Pf : nullptr, l1,
                                                                     Ms.qidx, Ms.p, Ms.nq1d, m0, m1, m2);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_face_sf(const Mesh& M, const T* W, const T* V, T* slots, bool jvp, const T* Pf,
                           cudaStream_t st) {
  if (M.kind != DG_MESH_STRUCTURED || M.d != 3 || !M.qidx) return cudaErrorNotSupported;
  return jvp ? run_face_sf<T, true>(M, W, V, slots, Pf, st) : run_face_sf<T, false>(M, W, V, slots, nullptr, st);
}
template cudaError_t launch_face_sf<double>(const Mesh&, const double*, const double*, double*, bool, const double*,
                                            cudaStream_t);
template cudaError_t launch_face_sf<float>(const Mesh&, const float*, const float*, float*, bool, const float*,
                                           cudaStream_t);

}  // namespace dgk
