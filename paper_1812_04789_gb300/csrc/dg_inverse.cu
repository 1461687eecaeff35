// Batched inverse of the element blocks for block Jacobi (Sec. 6.3: the
// element-block smoother's factorisation, here an explicit inverse so that
// every application is one dense mat-vec per element).
//
// Gauss-Jordan elimination in place with partial pivoting: at step k the pivot
// is the largest |A[i][k]| over the rows i not yet used as pivots (the lowest
// row index on ties).  Rows are never swapped; after the n steps the matrix R
// holds the inverse with permuted rows and columns,
//   X[step(i)][prow(j)] = R[i][j],
// where prow(k) is the pivot row of step k and step(i) the step at which row i
// was the pivot.  A zero pivot marks the status word (the block is singular)
// and the step continues with pivot 1.
//
// Blocks come row-major, bstride elements apart.  The inverse leaves
// column-major with leading dimension ld = inv_ld(nb) (rows padded to a
// 16-byte multiple with zeros), the layout the block-Jacobi apply streams,
// except from the in-place global-memory path, which leaves it row-major.
//
// block_inverse_reg_kernel (nb <= 16 R): 256 threads as a 16 x 16 grid;
// thread (ty, tx) keeps the R x R entries of rows ty + 16 a and columns
// tx + 16 b in registers for the whole elimination, so a step costs R^2 FMAs
// per thread plus two shared-memory vectors (the pivot row and column) and
// three barriers.  The permuted, transposed result is staged in shared memory
// and written out coalesced.
// block_inverse_kernel (larger blocks): the block in shared memory, one warp
// per row in the update.  block_inverse_panel_kernel (blocks that do not fit
// shared memory): panels of columns eliminated in shared memory, one rank-16
// update of the block's other columns per panel.
#include <algorithm>
#include <climits>

#include "dg_internal.h"

namespace dgk {

namespace {

int num_sms_inv() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// the pivot candidate (|value| larger, or equal with a lower row) of two
__device__ __forceinline__ bool better(float va, int ia, float vb, int ib) {
  return va > vb || (va == vb && ia < ib);
}
__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
  return va > vb || (va == vb && ia < ib);
}

template <class T, int R>
__global__ void __launch_bounds__(256, 1) block_inverse_reg_kernel(T* __restrict__ blocks, int nb,
                                                                   size_t bstride, long nblk, int* status) {
  constexpr int NP = 16 * R;
  __shared__ T colk[NP], prow[NP];
  __shared__ T cand_v[16], cand_s[16];
  __shared__ int cand_i[16];
  __shared__ int piv_row[NP], step_of[NP];
  __shared__ int s_p;
  __shared__ T s_piv;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);   // nb * ld output staging (column-major)
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int ld = inv_ld<T>(nb), nl = nb * ld;
  for (long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    T* Ag = blocks + (size_t)blk * bstride;
    T t[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) {
        const int i = ty + 16 * a, j = tx + 16 * b;
        t[a][b] = (i < nb && j < nb) ? Ag[(size_t)i * nb + j] : T(0);
      }
    unsigned used = 0;   // bit a: row ty + 16 a has been a pivot row
    bool bad = false;
    // k = 16 kb + kx: the register column kb is a compile-time index (the
    // unrolled kb loop), so reading and rewriting column k needs no selects
#pragma unroll
    for (int kb = 0; kb < R; ++kb)
    for (int kx = 0; kx < 16; ++kx) {
      const int k = 16 * kb + kx;
      if (k >= nb) break;
      T col[R];
#pragma unroll
      for (int a = 0; a < R; ++a) col[a] = t[a][kb];
      if (tx == kx) {   // the 16 owners of column k: best unused row of their R
        T best = T(-1), sv = T(0);
        int bi = INT_MAX;
#pragma unroll
        for (int a = 0; a < R; ++a) {
          const int i = ty + 16 * a;
          const T v = fabs(col[a]) >= T(0) ? fabs(col[a]) : T(0);   // NaN counts as 0
          if (i < nb && !((used >> a) & 1u) && better(v, i, best, bi)) {
            best = v;
            bi = i;
            sv = col[a];
          }
        }
        cand_v[ty] = best;
        cand_i[ty] = bi;
        cand_s[ty] = sv;
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        T v = l < 16 ? cand_v[l] : T(-1);
        int i = l < 16 ? cand_i[l] : INT_MAX;
        T sv = l < 16 ? cand_s[l] : T(0);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          const T v2 = __shfl_down_sync(0xffffffffu, v, o);
          const int i2 = __shfl_down_sync(0xffffffffu, i, o);
          const T s2 = __shfl_down_sync(0xffffffffu, sv, o);
          if (better(v2, i2, v, i)) {
            v = v2;
            i = i2;
            sv = s2;
          }
        }
        if (l == 0) {
          s_p = i;
          s_piv = sv;
          piv_row[k] = i;
          step_of[i] = k;
        }
      }
      __syncthreads();
      const int p = s_p, pa = p >> 4;
      T piv = s_piv;
      if (!(fabs(piv) > T(0))) {
        bad = true;
        piv = T(1);
      }
      const T ipiv = T(1) / piv;
      if (ty == (p & 15)) {   // the pivot row, scaled; its column k entry becomes 1 / piv
#pragma unroll
        for (int a = 0; a < R; ++a)
          if (a == pa) {
#pragma unroll
            for (int b = 0; b < R; ++b) {
              const int j = tx + 16 * b;
              if (j < NP) prow[j] = (j == k) ? ipiv : t[a][b] * ipiv;
            }
          }
        used |= 1u << pa;
      }
      if (tx == kx) {
#pragma unroll
        for (int a = 0; a < R; ++a) {
          const int i = ty + 16 * a;
          colk[i] = (i == p) ? T(0) : col[a];
        }
      }
      __syncthreads();
      T pr[R], ck[R];
#pragma unroll
      for (int b = 0; b < R; ++b) pr[b] = prow[tx + 16 * b];
#pragma unroll
      for (int a = 0; a < R; ++a) ck[a] = colk[ty + 16 * a];
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) t[a][b] -= ck[a] * pr[b];
      if (ty == (p & 15)) {
#pragma unroll
        for (int a = 0; a < R; ++a)
          if (a == pa) {
#pragma unroll
            for (int b = 0; b < R; ++b) t[a][b] = pr[b];
          }
      }
      if (tx == kx) {
#pragma unroll
        for (int a = 0; a < R; ++a) {
          const int i = ty + 16 * a;
          t[a][kb] = (i == p) ? ipiv : -ck[a] * ipiv;
        }
      }
    }
    __syncthreads();   // piv_row / step_of complete
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) {
        const int i = ty + 16 * a, j = tx + 16 * b;
        if (i < nb && j < nb) S[(size_t)piv_row[j] * ld + step_of[i]] = t[a][b];
      }
    for (int e = threadIdx.x; e < nb * (ld - nb); e += blockDim.x) {
      const int c = e / (ld - nb);
      S[(size_t)c * ld + nb + (e - c * (ld - nb))] = T(0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nl; e += blockDim.x) Ag[e] = S[e];
    if (bad && threadIdx.x == 0) atomicOr(status, ST_SINGULAR);
    __syncthreads();
  }
}

// Blocks too large for registers: the same elimination on a copy in shared
// memory (or in place in global memory).  One warp per row in the update.
template <class T>
__global__ void __launch_bounds__(256) block_inverse_kernel(T* __restrict__ blocks, int nb, size_t bstride,
                                                            long nblk, int use_smem, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // byte layout: colk[nb] | prow[nb] | piv_row[nb] | step_of[nb] | used[nb] | lead[nb] | A (16-aligned)
  T* colk = reinterpret_cast<T*>(smem_raw);
  T* prow = colk + nb;
  int* piv_row = reinterpret_cast<int*>(prow + nb);
  int* step_of = piv_row + nb;
  int* used = step_of + nb;
  int* lead = used + nb;
  __shared__ T wv[8], ws[8];
  __shared__ int wi[8];
  __shared__ int s_p;
  __shared__ T s_piv;
  T* As = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(lead + nb) + 15) & ~uintptr_t(15));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nn = nb * nb;
  const int ld = inv_ld<T>(nb);
  for (long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    T* Ag = blocks + (size_t)blk * bstride;
    T* A = use_smem ? As : Ag;
    if (use_smem)
      for (int e = threadIdx.x; e < nn; e += blockDim.x) A[e] = Ag[e];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) used[i] = 0;
    __syncthreads();
    bool bad = false;
    for (int k = 0; k < nb; ++k) {
      T best = T(-1), sv = T(0);
      int bi = INT_MAX;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const T x = A[(size_t)i * nb + k], v = fabs(x) >= T(0) ? fabs(x) : T(0);   // NaN counts as 0
        if (!used[i] && better(v, i, best, bi)) {
          best = v;
          bi = i;
          sv = x;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T v2 = __shfl_down_sync(0xffffffffu, best, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        const T s2 = __shfl_down_sync(0xffffffffu, sv, o);
        if (better(v2, i2, best, bi)) {
          best = v2;
          bi = i2;
          sv = s2;
        }
      }
      if (lane == 0) {
        wv[warp] = best;
        wi[warp] = bi;
        ws[warp] = sv;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
          if (better(wv[w], wi[w], best, bi)) {
            best = wv[w];
            bi = wi[w];
            sv = ws[w];
          }
        s_p = bi;
        s_piv = sv;
        piv_row[k] = bi;
        step_of[bi] = k;
        used[bi] = 1;
      }
      __syncthreads();
      const int p = s_p;
      T piv = s_piv;
      if (!(fabs(piv) > T(0))) {
        bad = true;
        piv = T(1);
      }
      const T ipiv = T(1) / piv;
      for (int j = threadIdx.x; j < nb; j += blockDim.x) prow[j] = (j == k) ? ipiv : A[(size_t)p * nb + j] * ipiv;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) colk[i] = (i == p) ? T(0) : A[(size_t)i * nb + k];
      __syncthreads();
      for (int i = warp; i < nb; i += nw) {
        T* row = A + (size_t)i * nb;
        const T c = colk[i];
        if (i == p) {
          for (int j = lane; j < nb; j += 32) row[j] = prow[j];
        } else {
          for (int j = lane; j < nb; j += 32) row[j] = (j == k) ? -c * ipiv : row[j] - c * prow[j];
        }
      }
      __syncthreads();
    }
    // permute into the output: X[step_of[i]][piv_row[j]] = R[i][j], column-major
    if (use_smem) {
      for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int i = e / nb, j = e - i * nb;
        Ag[(size_t)piv_row[j] * ld + step_of[i]] = A[e];
      }
      for (int e = threadIdx.x; e < nb * (ld - nb); e += blockDim.x) {
        const int c = e / (ld - nb);
        Ag[(size_t)c * ld + nb + (e - c * (ld - nb))] = T(0);
      }
    } else {
      // in place in global memory: the row permutation i -> step_of[i], then
      // the column permutation j -> piv_row[j], each applied cycle by cycle
      // (thread 0 marks every cycle's smallest index with the cycle length)
      for (int pass = 0; pass < 2; ++pass) {
        const int* to = pass == 0 ? step_of : piv_row;
        __syncthreads();
        if (threadIdx.x == 0) {
          for (int i = 0; i < nb; ++i) used[i] = 0;
          for (int i0 = 0; i0 < nb; ++i0) {
            lead[i0] = 0;
            if (used[i0]) continue;
            int c = i0, len = 0;
            do {
              used[c] = 1;
              c = to[c];
              ++len;
            } while (c != i0);
            lead[i0] = len > 1 ? len : 0;
          }
        }
        __syncthreads();
        for (int i0 = 0; i0 < nb; ++i0) {
          const int len = lead[i0];
          if (len == 0) continue;
          for (int x = threadIdx.x; x < nb; x += blockDim.x) {
            // pass 0 moves rows (x = column), pass 1 moves columns (x = row)
            const size_t str = pass == 0 ? (size_t)nb : 1, off = pass == 0 ? (size_t)x : (size_t)x * nb;
            T carry = A[off + (size_t)i0 * str];
            int src = i0;
            for (int s = 0; s < len; ++s) {
              const int dst = to[src];
              const T y = A[off + (size_t)dst * str];
              A[off + (size_t)dst * str] = carry;
              carry = y;
              src = dst;
            }
          }
        }
      }
    }
    if (bad && threadIdx.x == 0) atomicOr(status, ST_SINGULAR);
    __syncthreads();
  }
}

// Blocks too large for shared memory (nb = 420 at p = 6): Gauss-Jordan by
// panels of BP columns.  The BP elimination steps of a panel act on any other
// column x as x <- x + sum_c (X_c - e_{p_c}) x[p_c], where p_c is the pivot row
// of step c and X_c the panel's column c once the whole panel is eliminated
// (it is T e_{p_c}, T the product of the panel's steps: a GJ step changes a
// column only through its entry at the pivot row, and leaves e_i alone for a
// row i that is not the pivot).  So a panel is eliminated in shared memory
// (pivot search, the step on the panel's columns) and every other column of
// the block receives one rank-BP update, read and written once per panel
// instead of once per step.  Same pivot rule and in-place storage as above;
// the result is row-major, permuted in place at the end.
template <class T, int BP>
__global__ void __launch_bounds__(256) block_inverse_panel_kernel(T* __restrict__ blocks, int nb, size_t bstride,
                                                                  long nblk, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // byte layout: Pn[nb][BP] | piv_row[nb] | step_of[nb] | used[nb] | lead[nb]
  T* Pn = reinterpret_cast<T*>(smem_raw);
  int* piv_row = reinterpret_cast<int*>(Pn + (size_t)nb * BP);
  int* step_of = piv_row + nb;
  int* used = step_of + nb;
  int* lead = used + nb;
  __shared__ T wv[8], ws[8];
  __shared__ int wi[8];
  __shared__ int s_p;
  __shared__ T s_piv;
  __shared__ int pr[BP];          // pivot rows of the current panel
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    T* A = blocks + (size_t)blk * bstride;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) used[i] = 0;
    bool bad = false;
    for (int k0 = 0; k0 < nb; k0 += BP) {
      const int bw = min(BP, nb - k0);
      __syncthreads();
      for (int t = threadIdx.x; t < nb * BP; t += blockDim.x) {
        const int i = t / BP, c = t - i * BP;
        Pn[t] = c < bw ? A[(size_t)i * nb + k0 + c] : T(0);
      }
      __syncthreads();
      for (int c = 0; c < bw; ++c) {
        const int k = k0 + c;
        T best = T(-1), sv = T(0);
        int bi = INT_MAX;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
          const T x = Pn[(size_t)i * BP + c], v = fabs(x) >= T(0) ? fabs(x) : T(0);   // NaN counts as 0
          if (!used[i] && better(v, i, best, bi)) {
            best = v;
            bi = i;
            sv = x;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T v2 = __shfl_down_sync(0xffffffffu, best, o);
          const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
          const T s2 = __shfl_down_sync(0xffffffffu, sv, o);
          if (better(v2, i2, best, bi)) {
            best = v2;
            bi = i2;
            sv = s2;
          }
        }
        if (lane == 0) {
          wv[warp] = best;
          wi[warp] = bi;
          ws[warp] = sv;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          for (int w = 1; w < nw; ++w)
            if (better(wv[w], wi[w], best, bi)) {
              best = wv[w];
              bi = wi[w];
              sv = ws[w];
            }
          s_p = bi;
          s_piv = sv;
          piv_row[k] = bi;
          step_of[bi] = k;
          used[bi] = 1;
          pr[c] = bi;
        }
        __syncthreads();
        const int p = s_p;
        T piv = s_piv;
        if (!(fabs(piv) > T(0))) {
          bad = true;
          piv = T(1);
        }
        const T ipiv = T(1) / piv;
        // the step on the panel's columns, a thread per row i != p (the pivot
        // row keeps its old values until every other row has used them)
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
          if (i == p) continue;
          T* pi = Pn + (size_t)i * BP;
          const T* pp = Pn + (size_t)p * BP;
          const T m = pi[c];
          for (int cc = 0; cc < bw; ++cc) pi[cc] = cc == c ? -m * ipiv : pi[cc] - m * pp[cc] * ipiv;
        }
        __syncthreads();
        for (int cc = threadIdx.x; cc < bw; cc += blockDim.x)
          Pn[(size_t)p * BP + cc] = cc == c ? ipiv : Pn[(size_t)p * BP + cc] * ipiv;
        __syncthreads();
      }
      // every other column: x <- x + sum_c (X_c - e_{p_c}) x[p_c], a thread per column:
      // the panel rows X[i][0..BP) in 16-byte loads, then the e_{p_c} terms on the
      // panel's pivot rows (distinct rows, one subtraction each)
      for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        if (j >= k0 && j < k0 + bw) continue;
        T xp[BP];
#pragma unroll
        for (int c = 0; c < BP; ++c) xp[c] = c < bw ? A[(size_t)pr[c] * nb + j] : T(0);
        // eight rows' loads in flight before their updates
        int i = 0;
        for (; i + 8 <= nb; i += 8) {
          T a[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) a[u] = A[(size_t)(i + u) * nb + j];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            T pi[BP];
            ld_vec<T, BP>(Pn + (size_t)(i + u) * BP, pi);
            T acc = a[u];
#pragma unroll
            for (int c = 0; c < BP; ++c) acc += pi[c] * xp[c];
            A[(size_t)(i + u) * nb + j] = acc;
          }
        }
        for (; i < nb; ++i) {
          T pi[BP];
          ld_vec<T, BP>(Pn + (size_t)i * BP, pi);
          T acc = A[(size_t)i * nb + j];
#pragma unroll
          for (int c = 0; c < BP; ++c) acc += pi[c] * xp[c];
          A[(size_t)i * nb + j] = acc;
        }
#pragma unroll
        for (int c = 0; c < BP; ++c)
          if (c < bw) A[(size_t)pr[c] * nb + j] -= xp[c];
      }
      for (int t = threadIdx.x; t < nb * bw; t += blockDim.x) {
        const int i = t / bw, c = t - i * bw;
        A[(size_t)i * nb + k0 + c] = Pn[(size_t)i * BP + c];
      }
    }
    // in place: the row permutation i -> step_of[i], then the column
    // permutation j -> piv_row[j], each applied cycle by cycle
    for (int pass = 0; pass < 2; ++pass) {
      const int* to = pass == 0 ? step_of : piv_row;
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int i = 0; i < nb; ++i) used[i] = 0;
        for (int i0 = 0; i0 < nb; ++i0) {
          lead[i0] = 0;
          if (used[i0]) continue;
          int c = i0, len = 0;
          do {
            used[c] = 1;
            c = to[c];
            ++len;
          } while (c != i0 && len <= nb);
          lead[i0] = len > 1 ? len : 0;
        }
      }
      __syncthreads();
      for (int i0 = 0; i0 < nb; ++i0) {
        const int len = lead[i0];
        if (len == 0) continue;
        for (int x = threadIdx.x; x < nb; x += blockDim.x) {
          const size_t str = pass == 0 ? (size_t)nb : 1, off = pass == 0 ? (size_t)x : (size_t)x * nb;
          T carry = A[off + (size_t)i0 * str];
          int src = i0;
          for (int s = 0; s < len; ++s) {
            const int dst = to[src];
            const T y = A[off + (size_t)dst * str];
            A[off + (size_t)dst * str] = carry;
            carry = y;
            src = dst;
          }
        }
      }
    }
    if (bad && threadIdx.x == 0) atomicOr(status, ST_SINGULAR);
    __syncthreads();
  }
}

template <class T, int R>
cudaError_t run_reg(T* A, int nb, size_t bstride, long nblk, int* status, cudaStream_t st) {
  const size_t smem = (size_t)nb * inv_ld<T>(nb) * sizeof(T);
  if (smem > 48 * 1024)
    allow_max_smem(block_inverse_reg_kernel<T, R>);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, block_inverse_reg_kernel<T, R>, 256, smem);
  const long grid = std::min<long>(nblk, (long)std::max(1, occ) * num_sms_inv());
  note_launch();
  block_inverse_reg_kernel<T, R><<<(int)grid, 256, smem, st>>>(A, nb, bstride, nblk, status);
  return cudaGetLastError();
}

}  // namespace

template <class T>
cudaError_t launch_block_inverse(T* A, int nb, size_t bstride, long nblk, int* status, int* transposed,
                                 cudaStream_t st) {
  *transposed = 1;
  if (nblk <= 0) return cudaSuccess;
  // register tiles: R x R values of T per thread (at most 128 32-bit registers)
  const int R = (nb + 15) / 16;
  constexpr int RMAX = sizeof(T) == 4 ? 11 : 8;
  if (R <= RMAX) {
    if (R <= 1) return run_reg<T, 1>(A, nb, bstride, nblk, status, st);
    if (R <= 2) return run_reg<T, 2>(A, nb, bstride, nblk, status, st);
    if (R <= 4) return run_reg<T, 4>(A, nb, bstride, nblk, status, st);
    if (R <= 8) return run_reg<T, 8>(A, nb, bstride, nblk, status, st);
    return run_reg<T, (RMAX > 8 ? RMAX : 8)>(A, nb, bstride, nblk, status, st);
  }
  const int threads = 256;
  const size_t base = 2 * nb * sizeof(T) + 4 * nb * sizeof(int) + 32;
  const size_t full = base + (size_t)nb * nb * sizeof(T);
  int smax = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int use_smem = full <= (size_t)smax - 1024;
  if (!use_smem) {   // panels of 16 columns in shared memory, rank-16 updates of the rest in global memory
    constexpr int BP = 16;
    const size_t psm = (size_t)nb * BP * sizeof(T) + 4 * (size_t)nb * sizeof(int);
    if (psm <= (size_t)smax - 1024) {
      if (psm > 48 * 1024) allow_max_smem(block_inverse_panel_kernel<T, BP>);
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, block_inverse_panel_kernel<T, BP>, 256, psm);
      const long grid = std::min<long>(nblk, (long)std::max(1, occ) * num_sms_inv());
      *transposed = 0;
      note_launch();
      block_inverse_panel_kernel<T, BP><<<(int)grid, 256, psm, st>>>(A, nb, bstride, nblk, status);
      return cudaGetLastError();
    }
  }
  const size_t smem = use_smem ? full : base;
  if (smem > 48 * 1024)
    allow_max_smem(block_inverse_kernel<T>);
  const long grid = std::min<long>(nblk, (use_smem ? 1L : 8L) * num_sms_inv());
  *transposed = use_smem;
  note_launch();
  block_inverse_kernel<T><<<(int)grid, threads, smem, st>>>(A, nb, bstride, nblk, use_smem, status);
  return cudaGetLastError();
}
template cudaError_t launch_block_inverse<double>(double*, int, size_t, long, int*, int*, cudaStream_t);
template cudaError_t launch_block_inverse<float>(float*, int, size_t, long, int*, int*, cudaStream_t);

}  // namespace dgk
