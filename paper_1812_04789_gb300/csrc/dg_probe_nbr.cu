// Neighbour blocks of the first coarse level (Sec. 6.3: the inherited
// block-sparse operator needs dR_e/dW_nbr restricted to the coarse modes),
// FP32, for the mixed-precision preconditioner when the diagonal blocks come
// from the tensor-core probe.
//
// For face s of element e (neighbour n = nbr(e, s), which sees the face as its
// local face s ^ 1), with nmc coarse modes per variable:
//   O[(v,i'),(w,i)] = sum_q sum_c sum_s' Test_c(q, i') J_q[(v,c),(w,s')] TrialN_s'(q, i),
// J_q the derivative of the face-point outputs c (numerical flux, the two
// lifting integrands, the own dual tensor) with respect to the input s' (value,
// gradient components) of variable w on the neighbour's trace, Test_c the own
// face's weighted test functions (the same rows as the tensor-core probe's
// table) and TrialN the neighbour's basis on its face.  Per face and chunk of
// points: (J) one dual-number evaluation per (point, w, s'), (Z) the test side
// contracted first, Z[(w,v,i'), (q,s')] = sum_c Test J, (O) O += Z TrialN,
// summed in registers over the face's chunks and written to the block once.
// Faces of a direction with a single element are not handled here (they feed
// the diagonal block; the SIMT probe covers that case).
#include <algorithm>

#include "dg_probe.cuh"

namespace dgk {

namespace {

constexpr int NBR_THREADS = 256;
constexpr int NBR_ACC = 10;   // block entries a thread holds in registers across a face's point chunks

struct NbrPlan {
  int ok = 0, jq = 0, oFU = 0, oJ = 0, oT = 0, oN = 0, oZ = 0, smem = 0;
};

NbrPlan nbr_plan(int d, int nm, int nqf, int nmc, int smax) {
  NbrPlan P;
  const int M = d + 2, NF = 2 * d, KMX = 3 + d, PU = M * (1 + d), nb = M * nm, R = M * M * nmc;
  // about one thread per (point, seed variable, input) in the J phase
  int jq = std::max(1, std::min(nqf, NBR_THREADS / (M * 4)));
  for (; jq >= 1; jq = jq > 1 ? jq / 2 : 0) {
    long o = 0;
    auto take = [&](long n) {
      long r = o;
      o = (o + n + 3) / 4 * 4;
      return (int)r;
    };
    take((long)(1 + NF) * nb);                 // cW
    P.oFU = take((long)NF * 2 * nqf * PU);
    P.oJ = take((long)jq * M * 4 * M * KMX);
    P.oT = take((long)jq * KMX * nmc);
    P.oN = take((long)jq * 4 * nmc);
    P.oZ = take((long)jq * R * 4);
    if (o * (long)sizeof(float) <= smax) {
      P.jq = jq;
      P.smem = (int)(o * sizeof(float));
      P.ok = 1;
      return P;
    }
    if (jq == 1) break;
  }
  return P;
}

template <int D>
__global__ void __launch_bounds__(NBR_THREADS, 1) probe_nbr_kernel(MeshView<float> mv, Phys<float> ph,
                                                                const float* __restrict__ W,
                                                                float* __restrict__ Oout, int nmc, int ldo,
                                                                const float* __restrict__ test, int npv,
                                                                int nmp, NbrPlan P, int* status) {
  using T = float;
  constexpr int M = D + 2, NF = 2 * D, KMX = 3 + D, PU = M * (1 + D), NS = 1 + D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* cW = sm;
  T* cFU = sm + P.oFU;
  T* Jn = sm + P.oJ;   // [jq][w][4][v][c]
  T* Ts = sm + P.oT;   // [jq][c][nmc]
  T* Tn = sm + P.oN;   // [jq][4][nmc]
  T* Zs = sm + P.oZ;   // [jq][row][4], row = (w, v, i')
  const int nm = mv.nm, nqf = mv.nqf, E = mv.E, jq = P.jq;
  const int R = M * M * nmc, nbc = M * nmc;
  // ldo > 0: blocks column-major with leading dimension ldo, nbc * ldo apart;
  // ldo == 0: row-major, nbc * nbc apart
  const size_t ostride = ldo > 0 ? (size_t)nbc * ldo : (size_t)nbc * nbc;
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    int nbrs[NF];
#pragma unroll
    for (int s = 0; s < NF; ++s) nbrs[s] = mv.nbr[e * NF + s];
    probe_stage_primal<D, T>(mv, ph, W, e, nbrs, cW, nullptr, cFU, false, status);
    for (int s = 0; s < NF; ++s) {
      T* Os = Oout + ((size_t)e * NF + s) * ostride;
      const int f = s ^ 1;   // the neighbour's local face
      T oacc[NBR_ACC];
      for (int q0 = 0; q0 < nqf; q0 += jq) {
        const int ncj = min(jq, nqf - q0);
        // (J) neighbour-seeded tangents of the face-point outputs
        for (int t = threadIdx.x; t < ncj * M * 4; t += blockDim.x) {
          const int pl = t / (M * 4), w = (t >> 2) % M, sd = t & 3, q = q0 + pl;
          T* jo = Jn + (((size_t)pl * M + w) * 4 + sd) * M * KMX;
          if (sd < NS) {
            T sgo[D], sgn[D];
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
              sgo[kk] = T(0);
              sgn[kk] = sd == 1 + kk ? T(1) : T(0);
            }
            T oGL[M], oGR[M], oFp[M], oDo[M * D];
            face_point_tangent<D, T>(cFU + ((size_t)(s * 2) * nqf + q) * PU, cFU + ((size_t)(s * 2 + 1) * nqf + q) * PU,
                                     s / 2, s % 2, w, T(0), sgo, sd == 0 ? T(1) : T(0), sgn, ph, oGL, oGR, oFp,
                                     oDo);
#pragma unroll
            for (int v = 0; v < M; ++v) {
              jo[v * KMX + 0] = oFp[v];
              jo[v * KMX + 1] = oGL[v];
              jo[v * KMX + 2] = oGR[v];
#pragma unroll
              for (int kk = 0; kk < D; ++kk) jo[v * KMX + 3 + kk] = oDo[v * D + kk];
            }
          } else {
#pragma unroll
            for (int j = 0; j < M * KMX; ++j) jo[j] = T(0);
          }
        }
        // test rows of the own face and the neighbour's trial functions at the chunk's points
        for (int t = threadIdx.x; t < ncj * KMX * nmc; t += blockDim.x) {
          const int ip = t % nmc, c = (t / nmc) % KMX, pl = t / (nmc * KMX);
          Ts[t] = test[((size_t)(npv + s * nqf + q0 + pl) * KMX + c) * nmp + ip];
        }
        for (int t = threadIdx.x; t < ncj * 4 * nmc; t += blockDim.x) {
          const int i = t % nmc, sd = (t / nmc) % 4, pl = t / (4 * nmc), q = q0 + pl;
          T val = T(0);
          if (sd == 0)
            val = mv.fphi[((size_t)f * nqf + q) * nm + i];
          else if (sd < NS)
            val = mv.fdphi[(((size_t)f * D + (sd - 1)) * nqf + q) * nm + i];
          Tn[t] = val;
        }
        __syncthreads();
        // (Z) test side first
        for (int t = threadIdx.x; t < ncj * R; t += blockDim.x) {
          const int pl = t / R, row = t - pl * R;
          const int w = row / nbc, v = (row / nmc) % M, ip = row % nmc;
          const T* tr = Ts + (size_t)pl * KMX * nmc + ip;
          T tv[KMX];
#pragma unroll
          for (int c = 0; c < KMX; ++c) tv[c] = tr[c * nmc];
#pragma unroll
          for (int sd = 0; sd < 4; ++sd) {
            const T* jr = Jn + (((size_t)pl * M + w) * 4 + sd) * M * KMX + v * KMX;
            T z = T(0);
#pragma unroll
            for (int c = 0; c < KMX; ++c) z += tv[c] * jr[c];
            Zs[(size_t)t * 4 + sd] = z;
          }
        }
        __syncthreads();
        // (O) trial side: a thread's entries t = threadIdx.x + u * blockDim.x
        // accumulate in registers over the face's chunks (or, for blocks with
        // more than NBR_ACC * blockDim.x entries, in the block in global memory)
#pragma unroll
        for (int u = 0; u < NBR_ACC; ++u) {
          const int t = threadIdx.x + u * blockDim.x;
          if (t < R * nmc) {
            const int row = t / nmc, i = t - row * nmc;
            T a = T(0);
            for (int pl = 0; pl < ncj; ++pl) {
              const float4 z = *reinterpret_cast<const float4*>(Zs + ((size_t)pl * R + row) * 4);
              const T* tn = Tn + (size_t)pl * 4 * nmc + i;
              a += z.x * tn[0] + z.y * tn[nmc] + z.z * tn[2 * nmc] + z.w * tn[3 * nmc];
            }
            oacc[u] = q0 == 0 ? a : oacc[u] + a;
          }
        }
        for (int t = threadIdx.x + NBR_ACC * blockDim.x; t < R * nmc; t += blockDim.x) {
          const int row = t / nmc, i = t - row * nmc;
          const int w = row / nbc, v = (row / nmc) % M, ip = row % nmc;
          T acc = T(0);
          for (int pl = 0; pl < ncj; ++pl) {
            const T* z = Zs + ((size_t)pl * R + row) * 4;
            const T* tn = Tn + (size_t)pl * 4 * nmc + i;
#pragma unroll
            for (int sd = 0; sd < 4; ++sd) acc += z[sd] * tn[sd * nmc];
          }
          T* o = ldo > 0 ? Os + (size_t)(w * nmc + i) * ldo + v * nmc + ip
                         : Os + (size_t)(v * nmc + ip) * nbc + w * nmc + i;
          *o = q0 == 0 ? acc : *o + acc;
        }
        __syncthreads();
      }
      // the register-held entries of the face's block, written once
#pragma unroll
      for (int u = 0; u < NBR_ACC; ++u) {
        const int t = threadIdx.x + u * blockDim.x;
        if (t < R * nmc) {
          const int row = t / nmc, i = t - row * nmc;
          const int w = row / nbc, v = (row / nmc) % M, ip = row % nmc;
          T* o = ldo > 0 ? Os + (size_t)(w * nmc + i) * ldo + v * nmc + ip
                         : Os + (size_t)(v * nmc + ip) * nbc + w * nmc + i;
          *o = oacc[u];
        }
      }
    }
  }
}

int num_sms_nbr() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

bool probe_nbr_fits(const Mesh& M, int nmc) {
  if (!M.tc.ok || !M.tc_test || nmc < 1 || nmc > M.nm) return false;
  for (int k = 0; k < M.d; ++k)
    if (M.desc.n[k] == 1) return false;
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return nbr_plan(M.d, M.nm, M.nqf, nmc, smax).ok != 0;
}

cudaError_t launch_probe_nbr(const Mesh& M, const float* W, float* O, int nmc, int colmajor, cudaStream_t st) {
  const int ldo = colmajor ? inv_ld<float>((M.d + 2) * nmc) : 0;
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const NbrPlan P = nbr_plan(M.d, M.nm, M.nqf, nmc, smax);
  if (!P.ok || !M.tc.ok) return cudaErrorInvalidValue;
  cudaError_t e;
  int occ = 0;
  if (M.d == 2) {
    if ((e = allow_max_smem(probe_nbr_kernel<2>)) !=
        cudaSuccess)
      return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_nbr_kernel<2>, NBR_THREADS, P.smem);
  } else {
    if ((e = allow_max_smem(probe_nbr_kernel<3>)) !=
        cudaSuccess)
      return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_nbr_kernel<3>, NBR_THREADS, P.smem);
  }
  const int grid = std::min(M.E, std::max(1, occ) * num_sms_nbr());
  note_launch();
  if (M.d == 2)
    probe_nbr_kernel<2><<<grid, NBR_THREADS, P.smem, st>>>(M.view<float>(), M.phys_t<float>(), W, O, nmc, ldo,
                                                           M.tc_test, M.tc.npv, M.tc.nmp, P, M.status);
  else
    probe_nbr_kernel<3><<<grid, NBR_THREADS, P.smem, st>>>(M.view<float>(), M.phys_t<float>(), W, O, nmc, ldo,
                                                           M.tc_test, M.tc.npv, M.tc.nmp, P, M.status);
  return cudaGetLastError();
}

}  // namespace dgk
