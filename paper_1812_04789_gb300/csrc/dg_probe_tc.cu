// Element Jacobian blocks on the 5th-generation tensor cores (FP32 blocks of
// the mixed-precision preconditioner; Sec. 5.1 eq. ODEDG, Sec. 6.3).
//
// The diagonal block of element e is a sum over its volume points and the
// points of its own faces,
//   D[(v,i'),(w,i)] = sigma |J| delta + sum_p sum_s Z_p[(w,v,i'), s] Trial_s(p, i),
//   Z_p[(w,v,i'), s] = sum_c Test_c(p, i') J_p[(v,c),(w,s)],
// with J_p the pointwise derivative of the point outputs c (volume: the flux
// columns F[v][k]; face: numerical flux, the two lifting integrands, the dual
// tensor) with respect to the point input s (value, d gradient components) of
// variable w, Test_c the weighted test functions (BR2 lifting folded in) and
// Trial_s the basis values and gradients.  The second sum is a dense GEMM
//   D^T-part[(w,v,i'), i] = Z[(w,v,i'), K] Trial[i, K]^T,  K = (point, s),
// with an element-dependent A = Z (rows: seed variable, variable, test mode)
// and an element-independent B = Trial (rows: trial mode, padded to npad).
//
// One persistent CTA of 256 threads per SM walks over elements.  Per element
// and group of seed variables: for every chunk of jq points, (J) dual-number
// evaluations give J_p for the group's seeds; then per K step (two points,
// 8 K values) the threads form Z in shared memory in the MMA operand layout,
// split into TF32 hi + lo parts, and one thread issues the tcgen05 MMAs
// (hi*hi + hi*lo + lo*hi: FP32-level accuracy) into FP32 accumulators in
// TMEM.  A and B are double-buffered: the threads build K step k+1 while the
// tensor core runs K step k; an mbarrier, signalled by tcgen05.commit, says
// when a buffer may be overwritten.  The epilogue reads TMEM and writes the
// block rows (plus sigma |J| on the diagonal) once: no read-modify-write.
//
// Every wait is bounded: a wait that runs out sets ST_TIMEOUT in the status
// word, and the CTA leaves its loops together with the others (the decision
// is taken at a block-wide barrier before the buffer the MMAs read is written
// again), waits once more, bounded, for the MMAs it issued, frees its TMEM and
// returns.  If that second wait runs out as well, MMAs may still write the
// freed TMEM columns: the blocks of a handle whose status shows ST_TIMEOUT,
// and every tensor-core probe on the device after it, are untrusted until the
// stream is synchronised and the handle is set up again.
#include <algorithm>
#include <vector>

#include "dg_probe.cuh"
#include "dg_umma.cuh"

namespace dgk {

namespace {

constexpr int TC_PROD = 256;                        // operand producers (8 warps)
constexpr int TC_ISSUERS = 2;                       // warps whose lane 0 issues MMAs (alternate tiles)
constexpr int TC_THREADS = TC_PROD + 32 * TC_ISSUERS;
constexpr int TC_MAX_TILES = 8;
constexpr int TC_TMEM_COLS = 512;
constexpr long long TC_WAIT_LIMIT = 4000000000LL;   // SM cycles (about 2 s)

// ---------------------------------------------------------------- tables
// test[u][c][nmp]: u < npv volume points (u >= nq: padding, zero), then the
// own-face points (s, q); c < 3 + d output kinds.  trial[ks][hl][npad * 8]:
// the B operand of K step ks (points 2ks, 2ks + 1; K = 4 * point + s) in the
// core-matrix layout, hl = 0 the TF32-rounded value, hl = 1 the remainder.
template <int D>
__global__ void tc_tables_kernel(MeshView<float> mv, float half_eta, TcPlan P, float* __restrict__ test,
                                 float* __restrict__ trial) {
  constexpr int NF = 2 * D, KMX = 3 + D, NS = 1 + D;
  const int nm = mv.nm, nq = mv.nq, nqf = mv.nqf;
  const long npts = P.npv + (long)NF * nqf;
  const long stride = (long)gridDim.x * blockDim.x;
  const long ntest = npts * KMX * P.nmp;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < ntest; t += stride) {
    const int i = (int)(t % P.nmp), c = (int)((t / P.nmp) % KMX);
    const long u = t / ((long)P.nmp * KMX);
    float val = 0.f;
    if (i < nm) {
      if (u < nq) {
        if (c < D) val = -mv.vw[u] * mv.vdphi[((size_t)c * nq + u) * nm + i];
      } else if (u >= P.npv) {
        const int uf = (int)(u - P.npv), s = uf / nqf, q = uf % nqf;
        const float sg = (s % 2) ? 1.f : -1.f;
        const float fwq = mv.fw[(size_t)(s / 2) * nqf + q];
        if (c == 0)
          val = (sg * fwq) * mv.fphi[((size_t)s * nqf + q) * nm + i];
        else if (c < 3)
          val = (sg * half_eta) * mv.liftT[(((size_t)s * 2 + (c - 1)) * nqf + q) * nm + i];
        else
          val = (-fwq) * mv.fdphi[(((size_t)s * D + (c - 3)) * nqf + q) * nm + i];
      }
    }
    test[t] = val;
  }
  const int per = P.npad * 8;
  const long ntr = (long)P.nks * 2 * per;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < ntr; t += stride) {
    const int within = (int)(t % per), hl = (int)((t / per) % 2);
    const long ks = t / (2L * per);
    // invert the layout: within = (i / 8) * 64 + (k / 4) * 32 + (i % 8) * 4 + k % 4
    const int g = within / 64, rem = within % 64, pl = rem / 32, ii = (rem % 32) / 4, sd = rem % 4;
    const int i = g * 8 + ii;
    const long u = 2 * ks + pl;
    float val = 0.f;
    if (i < nm && sd < NS) {
      if (u < nq) {
        val = sd == 0 ? mv.vphi[(size_t)u * nm + i] : mv.vdphi[((size_t)(sd - 1) * nq + u) * nm + i];
      } else if (u >= P.npv) {
        const int uf = (int)(u - P.npv), s = uf / nqf, q = uf % nqf;
        val = sd == 0 ? mv.fphi[((size_t)s * nqf + q) * nm + i]
                      : mv.fdphi[(((size_t)s * D + (sd - 1)) * nqf + q) * nm + i];
      }
    }
    const float h = umma::tf32_rna(val);
    trial[t] = hl == 0 ? h : val - h;
  }
}

// ---------------------------------------------------------------- kernel
// Z rows of one thread for the K step of local points 2kk, 2kk + 1: the
// thread owns pair (wl, v) and test modes i' = i0, i0 + tpw, ...
template <int NK, int KMX, int M>
__device__ __forceinline__ void tc_produce(const float* __restrict__ Jb, const float* __restrict__ Ts,
                                           float* __restrict__ Ahi, float* __restrict__ Alo, int kk, int G,
                                           int wl, int v, int i0, int tpw, int nm, int nmp) {
  float jv[2][4][NK];
#pragma unroll
  for (int pl = 0; pl < 2; ++pl)
#pragma unroll
    for (int sd = 0; sd < 4; ++sd)
#pragma unroll
      for (int c = 0; c < NK; ++c)
        jv[pl][sd][c] = Jb[((((size_t)(2 * kk + pl) * G + wl) * M + v) * 4 + sd) * KMX + c];
  for (int ip = i0; ip < nm; ip += tpw) {
    float z[2][4];
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
      float tv[NK];
#pragma unroll
      for (int c = 0; c < NK; ++c) tv[c] = Ts[((size_t)(2 * kk + pl) * KMX + c) * nmp + ip];
#pragma unroll
      for (int sd = 0; sd < 4; ++sd) {
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < NK; ++c) a = fmaf(tv[c], jv[pl][sd][c], a);
        z[pl][sd] = a;
      }
    }
    const int r = (wl * M + v) * nm + ip, rr = r & 127;
    const int off = (r >> 7) * 1024 + (rr >> 3) * 64 + (rr & 7) * 4;
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
      float4 h, l;
      h.x = umma::tf32_rna(z[pl][0]); l.x = z[pl][0] - h.x;
      h.y = umma::tf32_rna(z[pl][1]); l.y = z[pl][1] - h.y;
      h.z = umma::tf32_rna(z[pl][2]); l.z = z[pl][2] - h.z;
      h.w = umma::tf32_rna(z[pl][3]); l.w = z[pl][3] - h.w;
      *reinterpret_cast<float4*>(Ahi + off + pl * 32) = h;
      *reinterpret_cast<float4*>(Alo + off + pl * 32) = l;
    }
  }
}

template <int D>
__global__ void __launch_bounds__(TC_THREADS, 1)
    probe_tc_kernel(MeshView<float> mv, Phys<float> ph, const float* __restrict__ W, float sigma,
                    float* __restrict__ Dout, size_t dstride, const float* __restrict__ test,
                    const float* __restrict__ trial, TcPlan P, int* status) {
  using namespace umma;
  constexpr int M = D + 2, NS = 1 + D, NF = 2 * D, KMX = 3 + D, PU = M * (1 + D);
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 16);
  float* A = reinterpret_cast<float*>(smem + P.oA);     // [2 buffers][hi, lo][tiles][1024]
  float* Bs = reinterpret_cast<float*>(smem + P.oB);    // [2 buffers][hi, lo][npad * 8]
  float* Jb = reinterpret_cast<float*>(smem + P.oJ);    // [jq][G][M][4][KMX]
  float* Ts = reinterpret_cast<float*>(smem + P.oT);    // [jq][KMX][nmp]
  float* cW = reinterpret_cast<float*>(smem + P.oW);
  float* cU = reinterpret_cast<float*>(smem + P.oU);
  float* cFU = reinterpret_cast<float*>(smem + P.oFU);
  const int nb = mv.nb, nm = mv.nm, nq = mv.nq, nqf = mv.nqf, E = mv.E;
  const int tiles = P.tiles, npad = P.npad, nmp = P.nmp, G = P.G, jq = P.jq;
  const int bufA = 2 * tiles * 1024, bufB = 2 * npad * 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float sdj = sigma * mv.detJ;

  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], TC_ISSUERS);   // one commit per issuing thread
    mbar_init(&mbar[1], TC_ISSUERS);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, (uint32_t)P.tmem_cols);
  for (int t = threadIdx.x; t < 2 * bufA; t += blockDim.x) A[t] = 0.f;
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_tf32(128, npad);
  uint32_t issued[2] = {0u, 0u}, waited[2] = {0u, 0u};

  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    int nbrs[NF];
#pragma unroll
    for (int s = 0; s < NF; ++s) nbrs[s] = mv.nbr[e * NF + s];
    probe_stage_primal<D, float>(mv, ph, W, e, nbrs, cW, cU, cFU, true, status);
    for (int g = 0; g < P.ngroups; ++g) {
      const int w0 = g * G, Gc = min(G, M - w0);
      const int npair = Gc * M, tpw = TC_PROD / npair, rows = npair * nm;
      const int tilesG = (rows + 127) >> 7;
      int ks = 0;
      // K step whose operands are complete but whose MMAs are not issued yet
      // (-1: none); lane 0 of each of the TC_ISSUERS warps after the producers
      // issues them for the tiles ti = its index (mod TC_ISSUERS), each tile's
      // three passes in order (hi.hi, hi.lo, lo.hi), and commits once
      int pend = -1;
      auto issue_pending = [&]() {
        if (pend < 0) return;
        const int pb = pend & 1;
        const int is = ((int)threadIdx.x - TC_PROD) >> 5;
        if ((int)threadIdx.x >= TC_PROD && (threadIdx.x & 31) == 0) {
          fence_after_sync();
          const float* Ab = A + pb * bufA;
          const float* Bb = Bs + pb * bufB;
          const uint64_t bh = desc_kmajor(smem_u32(Bb)), bl = desc_kmajor(smem_u32(Bb + npad * 8));
#pragma unroll 1
          for (int ti = is; ti < tilesG; ti += TC_ISSUERS) {
            const uint64_t ahi = desc_kmajor(smem_u32(Ab + ti * 1024));
            const uint64_t alo = desc_kmajor(smem_u32(Ab + tiles * 1024 + ti * 1024));
            const uint32_t d = tmem + (uint32_t)(ti * npad);
            mma_tf32(d, ahi, bh, idesc, pend > 0);
            mma_tf32(d, ahi, bl, idesc, true);
            mma_tf32(d, alo, bh, idesc, true);
          }
          commit(&mbar[pb]);
        }
        ++issued[pb];
        pend = -1;
      };
      // the B operand (bufB / 4 <= 4 npad <= 1024 float4) of the next K step, in registers
      constexpr int BPRE = (4 * 256 + TC_THREADS - 1) / TC_THREADS;
      float4 bpre[BPRE];
#pragma unroll
      for (int u = 0; u < BPRE; ++u) {
        const int t = threadIdx.x + u * TC_THREADS;
        bpre[u] = t < bufB / 4 ? reinterpret_cast<const float4*>(trial)[t] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int part = 0; part < 2; ++part) {
        const int npts = part == 0 ? P.npv : NF * nqf, ubase = part == 0 ? 0 : P.npv;
        for (int c0 = 0; c0 < npts; c0 += jq) {
          const int ncj = min(jq, npts - c0);   // even: npv and NF * nqf are
          // (J) pointwise derivatives for the group's seeds (w, s); s = NS pads to 4
          for (int t = threadIdx.x; t < ncj * Gc * 4; t += blockDim.x) {
            const int pl = t / (Gc * 4), wl = (t >> 2) % Gc, sd = t & 3, w = w0 + wl;
            float* jo = Jb + (((size_t)pl * G + wl) * M) * 4 * KMX + sd * KMX;   // + v * 4 * KMX + c
            if (part == 0) {
              const int u = c0 + pl;
              if (u < nq && sd < NS) {
                using S = Dual<float>;
                const float* pu = cU + (size_t)u * PU;
                S uu[M], gg[M][D], F[M][D];
#pragma unroll
                for (int v = 0; v < M; ++v) {
                  uu[v] = S(pu[v], (v == w && sd == 0) ? 1.f : 0.f);
#pragma unroll
                  for (int kk = 0; kk < D; ++kk)
                    gg[v][kk] = S(pu[M + v * D + kk], (v == w && sd == 1 + kk) ? 1.f : 0.f);
                }
                flux_total<D, S, float>(uu, gg, F, ph);
#pragma unroll
                for (int v = 0; v < M; ++v)
#pragma unroll
                  for (int kk = 0; kk < D; ++kk) jo[v * 4 * KMX + kk] = F[v][kk].d;
              } else {
#pragma unroll
                for (int v = 0; v < M; ++v)
#pragma unroll
                  for (int kk = 0; kk < D; ++kk) jo[v * 4 * KMX + kk] = 0.f;
              }
            } else {
              const int uf = c0 + pl, s = uf / nqf, q = uf % nqf;
              if (sd < NS) {
                float sgo[D], sgn[D];
#pragma unroll
                for (int kk = 0; kk < D; ++kk) {
                  sgo[kk] = sd == 1 + kk ? 1.f : 0.f;
                  sgn[kk] = 0.f;
                }
                float oGL[M], oGR[M], oFp[M], oDo[M * D];
                face_point_tangent<D, float>(cFU + ((size_t)(s * 2) * nqf + q) * PU,
                                             cFU + ((size_t)(s * 2 + 1) * nqf + q) * PU, s / 2, s % 2, w,
                                             sd == 0 ? 1.f : 0.f, sgo, 0.f, sgn, ph, oGL, oGR, oFp, oDo);
#pragma unroll
                for (int v = 0; v < M; ++v) {
                  jo[v * 4 * KMX + 0] = oFp[v];
                  jo[v * 4 * KMX + 1] = oGL[v];
                  jo[v * 4 * KMX + 2] = oGR[v];
#pragma unroll
                  for (int kk = 0; kk < D; ++kk) jo[v * 4 * KMX + 3 + kk] = oDo[v * D + kk];
                }
              } else {
#pragma unroll
                for (int v = 0; v < M; ++v)
#pragma unroll
                  for (int c = 0; c < KMX; ++c) jo[v * 4 * KMX + c] = 0.f;
              }
            }
          }
          {   // test rows of the chunk's points
            const float4* src = reinterpret_cast<const float4*>(test + (size_t)(ubase + c0) * KMX * nmp);
            float4* dst = reinterpret_cast<float4*>(Ts);
            for (int t = threadIdx.x; t < ncj * KMX * nmp / 4; t += blockDim.x) dst[t] = src[t];
          }
          __syncthreads();
          for (int kk = 0; kk < ncj / 2; ++kk, ++ks) {
            const int b = ks & 1;
            bool late = false;
            if (issued[b] > waited[b]) {   // the MMAs that last read buffer b (K step ks - 2)
              if (mbar_wait(&mbar[b], (issued[b] - 1u) & 1u, TC_WAIT_LIMIT))
                waited[b] = issued[b];
              else
                late = true;
            }
            // decided by the whole CTA before buffer b is written again: after a
            // wait that ran out, no thread touches operands the MMAs may still read
            if (__syncthreads_or(late)) {
              if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
              goto done;
            }
            issue_pending();   // K step ks - 1 (its operands complete at the barrier above)
#pragma unroll
            for (int u = 0; u < BPRE; ++u) {   // B of this step from registers, then prefetch the next
              const int t = threadIdx.x + u * TC_THREADS;
              if (t < bufB / 4) {
                reinterpret_cast<float4*>(Bs + b * bufB)[t] = bpre[u];
                if (ks + 1 < P.nks) bpre[u] = reinterpret_cast<const float4*>(trial + (size_t)(ks + 1) * bufB)[t];
              }
            }
            if ((int)threadIdx.x < npair * tpw) {
              const int pair = threadIdx.x / tpw, i0 = threadIdx.x % tpw;
              float* Ahi = A + b * bufA;
              if (part == 0)
                tc_produce<D, KMX, M>(Jb, Ts, Ahi, Ahi + tiles * 1024, kk, G, pair / M, pair % M, i0, tpw, nm,
                                      nmp);
              else
                tc_produce<KMX, KMX, M>(Jb, Ts, Ahi, Ahi + tiles * 1024, kk, G, pair / M, pair % M, i0, tpw,
                                        nm, nmp);
            }
            fence_proxy_async();
            pend = ks;
          }
          // the chunk's last operands are complete and Jb / Ts may be refilled
          // once every producer is here; its MMAs run during the next J stage
          __syncthreads();
          issue_pending();
        }
      }
      {   // drain, then the epilogue: TMEM -> block rows (v, i'), columns (w, i)
        bool late = false;
        for (int b = 0; b < 2; ++b)
          if (issued[b] > waited[b]) {
            if (mbar_wait(&mbar[b], (issued[b] - 1u) & 1u, TC_WAIT_LIMIT))
              waited[b] = issued[b];
            else
              late = true;
          }
        if (__syncthreads_or(late)) {
          if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
          goto done;
        }
        fence_after_sync();
        const int lb = (warp & 3) * 32;
        for (int ti = warp >> 2; warp < TC_PROD / 32 && ti < tilesG; ti += TC_PROD / 128) {
          const int r = ti * 128 + lb + lane;
          for (int c0 = 0; c0 < nm; c0 += 16) {
            float v16[16];
            tmem_ld16(tmem + ((uint32_t)lb << 16) + (uint32_t)(ti * npad + c0), v16);
            if (r < rows) {
              const int pair = r / nm, ip = r - pair * nm, w = w0 + pair / M, v = pair % M;
              float* drow = Dout + (size_t)e * dstride + (size_t)(v * nm + ip) * nb + (size_t)w * nm;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int i = c0 + j;
                if (i < nm) drow[i] = v16[j] + ((v == w && ip == i) ? sdj : 0.f);
              }
            }
          }
        }
        fence_before_sync();
        __syncthreads();
      }
    }
  }
done:
  // after a wait that ran out, MMAs may still be in flight: wait for them once
  // more (bounded) before the TMEM they write is freed for the next CTA
  for (int b = 0; b < 2; ++b)
    if (issued[b] > waited[b] && mbar_wait(&mbar[b], (issued[b] - 1u) & 1u, TC_WAIT_LIMIT)) waited[b] = issued[b];
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)P.tmem_cols);
}

int num_sms_tc() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

// ---------------------------------------------------------------- host
TcPlan tc_plan(int d, int nm, int nq, int nqf, int smem_max) {
  TcPlan P;
  const int M = d + 2, NF = 2 * d, KMX = 3 + d, PU = M * (1 + d), nb = M * nm;
  P.npad = (nm + 15) / 16 * 16;
  if (P.npad > 256) return P;
  P.nmp = (nm + 3) / 4 * 4;
  P.npv = (nq + 1) / 2 * 2;
  P.nks = (P.npv + NF * nqf) / 2;
  for (int G = M; G >= 1 && !P.G; --G) {
    const int tiles = (G * M * nm + 127) / 128;
    if (tiles <= TC_MAX_TILES && tiles * P.npad <= TC_TMEM_COLS) P.G = G;
  }
  if (!P.G) return P;
  P.tiles = (P.G * M * nm + 127) / 128;
  P.ngroups = (M + P.G - 1) / P.G;
  P.tmem_cols = 32;
  while (P.tmem_cols < P.tiles * P.npad) P.tmem_cols *= 2;
  for (int jq = 16; jq >= 2; jq /= 2) {
    long o = 128;   // two mbarriers and the TMEM address
    auto take = [&](long bytes) {
      long r = o;
      o = (o + bytes + 127) / 128 * 128;
      return (int)r;
    };
    P.oA = take(2L * 2 * P.tiles * 4096);
    P.oB = take(2L * 2 * P.npad * 32);
    P.oJ = take((long)jq * P.G * M * 4 * KMX * 4);
    P.oT = take((long)jq * KMX * P.nmp * 4);
    P.oW = take((long)(1 + NF) * nb * 4);
    P.oU = take((long)nq * PU * 4);
    P.oFU = take((long)NF * 2 * nqf * PU * 4);
    if (o <= smem_max) {
      P.jq = jq;
      P.smem = (int)o;
      P.ok = 1;
      return P;
    }
  }
  return P;
}

cudaError_t build_tc_tables(Mesh& M) {
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  M.tc = tc_plan(M.d, M.nm, M.nq, M.nqf, smax);
  if (!M.tc.ok) return cudaSuccess;
  const int KMX = 3 + M.d;
  const size_t ntest = ((size_t)M.tc.npv + 2 * M.d * M.nqf) * KMX * M.tc.nmp;
  const size_t ntrial = (size_t)M.tc.nks * 2 * M.tc.npad * 8;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&M.tc_test, ntest * sizeof(float))) != cudaSuccess) return e;
  M.allocs.push_back(M.tc_test);
  if ((e = cudaMalloc((void**)&M.tc_trial, ntrial * sizeof(float))) != cudaSuccess) return e;
  M.allocs.push_back(M.tc_trial);
  const float half_eta = 0.5f * M.phys_t<float>().eta;
  note_launch();
  if (M.d == 2)
    tc_tables_kernel<2><<<256, 256>>>(M.view<float>(), half_eta, M.tc, M.tc_test, M.tc_trial);
  else
    tc_tables_kernel<3><<<256, 256>>>(M.view<float>(), half_eta, M.tc, M.tc_test, M.tc_trial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaStreamSynchronize(0);
}

template <int D>
static cudaError_t run_tc(const Mesh& M, const float* W, float sigma, float* Dout, size_t dstride,
                          cudaStream_t st) {
  const TcPlan& P = M.tc;
  // at most 512 / tmem_cols co-resident CTAs per SM may hold TMEM at once:
  // request enough shared memory that no more fit
  const int per_sm = std::max(1, std::min(TC_TMEM_COLS / P.tmem_cols, 2048 / TC_THREADS));
  int smem = P.smem;
  const int sm_total = 228 * 1024;
  if (per_sm < 8) smem = std::max(smem, sm_total / (per_sm + 1) - 1024 + 16);
  cudaError_t e = allow_max_smem(probe_tc_kernel<D>);
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_tc_kernel<D>, TC_THREADS, smem);
  occ = std::max(1, std::min(occ, per_sm));
  const int grid = std::min(M.E, num_sms_tc() * occ);
  note_launch();
  probe_tc_kernel<D><<<grid, TC_THREADS, smem, st>>>(M.view<float>(), M.phys_t<float>(), W, sigma, Dout,
                                                     dstride, M.tc_test, M.tc_trial, P, M.status);
  return cudaGetLastError();
}

cudaError_t launch_probe_tc(const Mesh& M, const float* W, float sigma, float* D, size_t dstride,
                            cudaStream_t st) {
  if (!M.tc.ok) return cudaErrorInvalidValue;
  return M.d == 2 ? run_tc<2>(M, W, sigma, D, dstride, st) : run_tc<3>(M, W, sigma, D, dstride, st);
}

}  // namespace dgk
