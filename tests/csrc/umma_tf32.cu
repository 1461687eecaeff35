// Standalone check of the tcgen05 helpers in dg_umma.cuh: C (128 x N) =
// A (128 x K) B (N x K)^T on the tensor core with K-major no-swizzle operands,
// in one TF32 pass and in three passes (hi*hi + hi*lo + lo*hi), against a
// double-precision product on the host.  N covers the padded widths the block
// probe uses.  Exit status 0 when every case meets its bound.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "dg_umma.cuh"

using namespace dgk;

constexpr int MT = 128, K = 24, KS = K / 8;

template <int N>
__global__ void __launch_bounds__(128) gemm(const float* A, const float* B, float* C1, float* C3, int* err) {
  __shared__ __align__(128) float sA[2][KS][MT * 8];
  __shared__ __align__(128) float sB[2][KS][N * 8];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t slot;
  for (int t = threadIdx.x; t < MT * K; t += blockDim.x) {
    const int r = t / K, k = t % K;
    const float a = A[t], h = umma::tf32_rna(a);
    sA[0][k / 8][umma::tile_offset(r, k % 8)] = h;
    sA[1][k / 8][umma::tile_offset(r, k % 8)] = a - h;
  }
  for (int t = threadIdx.x; t < N * K; t += blockDim.x) {
    const int r = t / K, k = t % K;
    const float b = B[t], h = umma::tf32_rna(b);
    sB[0][k / 8][umma::tile_offset(r, k % 8)] = h;
    sB[1][k / 8][umma::tile_offset(r, k % 8)] = b - h;
  }
  if (threadIdx.x == 0) {
    umma::mbar_init(&mbar, 1);
    umma::fence_mbar_init();
  }
  constexpr uint32_t NCOL = N <= 32 ? 64 : (N <= 64 ? 128 : 256);
  if (threadIdx.x < 32) umma::tmem_alloc(&slot, NCOL);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tm = slot;
  const uint32_t c3 = NCOL / 2;   // second accumulator's first column
  if (threadIdx.x == 0) {
    const uint32_t id = umma::idesc_tf32(MT, N);
    for (int ks = 0; ks < KS; ++ks) {
      const uint64_t ah = umma::desc_kmajor(umma::smem_u32(sA[0][ks]));
      const uint64_t al = umma::desc_kmajor(umma::smem_u32(sA[1][ks]));
      const uint64_t bh = umma::desc_kmajor(umma::smem_u32(sB[0][ks]));
      const uint64_t bl = umma::desc_kmajor(umma::smem_u32(sB[1][ks]));
      umma::mma_tf32(tm, ah, bh, id, ks > 0);
      umma::mma_tf32(tm + c3, ah, bh, id, ks > 0);
      umma::mma_tf32(tm + c3, ah, bl, id, true);
      umma::mma_tf32(tm + c3, al, bh, id, true);
    }
    umma::commit(&mbar);
  }
  if (!umma::mbar_wait(&mbar, 0, 2000000000LL)) atomicOr(err, 1);
  umma::fence_after_sync();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r = warp * 32 + lane;
  for (int c0 = 0; c0 < N; c0 += 16) {
    float v[16];
    umma::tmem_ld16(tm + ((uint32_t)(warp * 32) << 16) + c0, v);
    for (int j = 0; j < 16; ++j) C1[r * N + c0 + j] = v[j];
    umma::tmem_ld16(tm + ((uint32_t)(warp * 32) << 16) + c3 + c0, v);
    for (int j = 0; j < 16; ++j) C3[r * N + c0 + j] = v[j];
  }
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) umma::tmem_dealloc(tm, NCOL);
}

template <int N>
static int run(std::mt19937_64& g) {
  std::uniform_real_distribution<float> U(-1.f, 1.f);
  std::vector<float> A(MT * K), B(N * K), C1(MT * N), C3(MT * N);
  for (auto& x : A) x = U(g);
  for (auto& x : B) x = U(g);
  float *dA, *dB, *dC1, *dC3;
  int* derr;
  cudaMalloc(&dA, A.size() * 4);
  cudaMalloc(&dB, B.size() * 4);
  cudaMalloc(&dC1, C1.size() * 4);
  cudaMalloc(&dC3, C3.size() * 4);
  cudaMalloc(&derr, 4);
  cudaMemset(derr, 0, 4);
  cudaMemcpy(dA, A.data(), A.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, B.data(), B.size() * 4, cudaMemcpyHostToDevice);
  gemm<N><<<1, 128>>>(dA, dB, dC1, dC3, derr);
  cudaError_t ce = cudaDeviceSynchronize();
  int herr = 0;
  cudaMemcpy(C1.data(), dC1, C1.size() * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(C3.data(), dC3, C3.size() * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC1);
  cudaFree(dC3);
  cudaFree(derr);
  if (ce != cudaSuccess) {
    printf("N=%d: CUDA error %s\n", N, cudaGetErrorString(ce));
    return 1;
  }
  // errors relative to sum_k |a_rk b_ck| (the natural scale of a dot product)
  double e1 = 0, e3 = 0;
  for (int r = 0; r < MT; ++r)
    for (int c = 0; c < N; ++c) {
      double s = 0, sa = 0;
      for (int k = 0; k < K; ++k) {
        s += (double)A[r * K + k] * B[c * K + k];
        sa += std::fabs((double)A[r * K + k] * B[c * K + k]);
      }
      e1 = std::fmax(e1, std::fabs(C1[r * N + c] - s) / sa);
      e3 = std::fmax(e3, std::fabs(C3[r * N + c] - s) / sa);
    }
  // one TF32 pass: operand rounding 2^-11 each; three passes: FP32-level
  const bool ok = herr == 0 && e1 < 2e-3 && e1 > 1e-6 && e3 < 2e-6;
  printf("N=%3d  timeout=%d  1-pass rel err %.3e  3-pass rel err %.3e  %s\n", N, herr, e1, e3, ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}

int main() {
  std::mt19937_64 g(1812);
  int bad = 0;
  bad += run<16>(g);
  bad += run<48>(g);
  bad += run<96>(g);
  return bad ? 1 : 0;
}
