// Element block ILU(0) of the coarsest p-multigrid level: the preconditioner
// of the coarsest smoother in Table MGSettings (Sec. 6.3: incomplete LU with
// zero fill on the element block pattern, in minimum-discarded-fill order).
//
// Matrix: the inherited coarse operator, A_ii = D_i (self couplings through a
// one-element periodic direction are already in D_i) and A_ij = the sum of
// i's face blocks towards j.  With no triangle in the face graph (no periodic
// direction of exactly three elements) ILU(0) never changes an off-diagonal
// block, so the factors are L_ik = A_ik S_k^{-1}, U_ij = A_ij and the pivot
// blocks
//     S_i = A_ii - sum_{k before i} A_ik S_k^{-1} A_ki,
// and only S_i^{-1} is stored.  Substitutions:
//     forward   y_i = S_i^{-1} (r_i - sum_{k before i} A_ik y_k)
//     backward  z_i = y_i - S_i^{-1} sum_{j after i} A_ij z_j.
// Rows of one level (no two of them neighbours) are independent: both the
// factorisation and the substitutions run level by level in ONE thread block
// (levels separated by __syncthreads; no wait on another block), the order
// and levels coming from the host (dg_bilu_order).
#include <algorithm>
#include <cmath>
#include <queue>
#include <vector>

#include "dg_internal.h"

namespace dgk {

// ------------------------------------------------------------ host ordering
namespace {

struct Graph {
  std::vector<std::vector<int>> nb;     // distinct neighbours (no self), ascending
  std::vector<std::vector<double>> c;   // c(i, nb[i][t])
};

int build_graph(int E, int nf, const int* nbr, const double* cin, Graph& g) {
  g.nb.assign(E, {});
  g.c.assign(E, {});
  for (int e = 0; e < E; ++e) {
    std::vector<std::pair<int, double>> l;
    for (int s = 0; s < nf; ++s) {
      const int k = nbr[(size_t)e * nf + s];
      if (k < 0 || k >= E) return -1;
      if (k == e) continue;
      bool seen = false;
      for (auto& q : l) seen = seen || q.first == k;
      if (!seen) l.push_back({k, cin ? cin[(size_t)e * nf + s] : 0.0});
    }
    std::sort(l.begin(), l.end());
    for (auto& q : l) {
      g.nb[e].push_back(q.first);
      g.c[e].push_back(q.second);
    }
  }
  return 0;
}

bool adjacent(const Graph& g, int a, int b) {
  for (int x : g.nb[a])
    if (x == b) return true;
  return false;
}

double cval(const Graph& g, int a, int b) {
  for (size_t t = 0; t < g.nb[a].size(); ++t)
    if (g.nb[a][t] == b) return g.c[a][t];
  return 0.0;
}

void order_mdf(const Graph& g, std::vector<int>& order) {
  const int E = (int)g.nb.size();
  std::vector<char> done(E, 0);
  auto weight = [&](int i) {
    double s = 0.0;
    for (int j : g.nb[i]) {
      if (done[j]) continue;
      for (int k : g.nb[i]) {
        if (done[k] || j == k || adjacent(g, j, k)) continue;
        const double f = cval(g, j, i) * cval(g, i, k);
        s += f * f;
      }
    }
    return std::sqrt(s);
  };
  std::vector<double> w(E);
  using Item = std::pair<double, int>;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
  for (int i = 0; i < E; ++i) {
    w[i] = weight(i);
    heap.push({w[i], i});
  }
  order.clear();
  while (!heap.empty()) {
    const Item it = heap.top();
    heap.pop();
    const int i = it.second;
    if (done[i] || it.first != w[i]) continue;   // stale entry
    done[i] = 1;
    order.push_back(i);
    for (int j : g.nb[i])
      if (!done[j]) {
        w[j] = weight(j);
        heap.push({w[j], j});
      }
  }
}

void order_colour(const Graph& g, std::vector<int>& order) {
  const int E = (int)g.nb.size();
  std::vector<int> col(E, 0);
  for (int i = 0; i < E; ++i) {
    std::vector<char> used(g.nb[i].size() + 1, 0);
    for (int j : g.nb[i])
      if (j < i && col[j] < (int)used.size()) used[col[j]] = 1;
    int c = 0;
    while (used[c]) ++c;
    col[i] = c;
  }
  order.resize(E);
  for (int i = 0; i < E; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return col[a] < col[b]; });
}

}  // namespace

int bilu_order_host(int E, int nf, const int* nbr, const double* c, int kind, int* order, int* level) {
  Graph g;
  if (E < 1 || nf < 0 || !nbr || !order || !level) return -1;
  if (kind == DG_ORDER_MDF && !c) return -1;
  if (build_graph(E, nf, nbr, kind == DG_ORDER_MDF ? c : nullptr, g) != 0) return -1;
  std::vector<int> o;
  if (kind == DG_ORDER_MDF) {
    order_mdf(g, o);
  } else if (kind == DG_ORDER_NATURAL) {
    o.resize(E);
    for (int i = 0; i < E; ++i) o[i] = i;
  } else if (kind == DG_ORDER_COLOUR) {
    order_colour(g, o);
  } else {
    return -1;
  }
  std::vector<int> pos(E);
  for (int p = 0; p < E; ++p) pos[o[p]] = p;
  int nlev = 0;
  for (int p = 0; p < E; ++p) {
    const int i = o[p];
    int l = 0;
    for (int k : g.nb[i])
      if (pos[k] < p) l = std::max(l, level[k] + 1);
    level[i] = l;
    nlev = std::max(nlev, l + 1);
    order[p] = i;
  }
  return nlev;
}

// ------------------------------------------------------------ device side
namespace {

template <class T>
__device__ __forceinline__ T blk(const T* b, int co_t, int ld, int nb, int r, int c) {
  return co_t ? b[(size_t)c * ld + r] : b[(size_t)r * nb + c];
}

// c[e][s] = ||A_ee^{-1} A_e,nbr(e,s)||_F for the first face of each distinct
// neighbour (the MDF weights' reduced matrix), -1 elsewhere.  One warp per
// (element, face); A_ee^{-1} is the block-Jacobi inverse of the level.
template <class T>
__global__ void __launch_bounds__(256) bilu_weights_kernel(const T* __restrict__ Dinv, size_t bs, int inv_t,
                                                           const T* __restrict__ O, size_t cs, int co_t,
                                                           const int* __restrict__ nbr, int nf, int nb, int E,
                                                           double* __restrict__ c) {
  const int lane = threadIdx.x & 31;
  const long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  if (w >= (long)E * nf) return;   // whole warps
  const int e = (int)(w / nf), s = (int)(w - (long)e * nf);
  const int k = nbr[(size_t)e * nf + s];
  bool first = k != e;
  for (int s2 = 0; s2 < s; ++s2) first = first && nbr[(size_t)e * nf + s2] != k;
  if (!first) {
    if (lane == 0) c[w] = -1.0;
    return;
  }
  const int ld = inv_ld<T>(nb);
  const T* Di = Dinv + (size_t)e * bs;
  double acc = 0.0;
  for (int t = lane; t < nb * nb; t += 32) {
    const int r = t / nb, col = t - r * nb;
    T x = T(0);
    for (int q = 0; q < nb; ++q) {
      T a = T(0);
      for (int s2 = s; s2 < nf; ++s2)
        if (nbr[(size_t)e * nf + s2] == k) a += blk(O + ((size_t)e * nf + s2) * cs, co_t, ld, nb, q, col);
      x += blk(Di, inv_t, ld, nb, r, q) * a;
    }
    acc += (double)x * (double)x;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) c[w] = sqrt(acc);
}

// Pivot blocks S_i and their inverses, level by level; one warp per element,
// three nb x nb scratch blocks per warp in shared memory.
template <class T>
__global__ void __launch_bounds__(1024) bilu_factor_kernel(const T* __restrict__ Dop, const T* __restrict__ O,
                                                           size_t cs, int co_t, const int* __restrict__ nbr,
                                                           int nf, const int* __restrict__ pos,
                                                           const int* __restrict__ lptr,
                                                           const int* __restrict__ lel,
                                                           const int* __restrict__ nlev_p, T* Sinv, int* status,
                                                           int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int ld = inv_ld<T>(nb), nb2 = nb * nb;
  T* S = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 3 * nb2;
  T* X = S + nb2;
  T* Y = X + nb2;
  const int nlev = *nlev_p;
  for (int lv = 0; lv < nlev; ++lv) {
    const int beg = lptr[lv], end = lptr[lv + 1];
    for (int idx = beg + warp; idx < end; idx += nw) {
      const int i = lel[idx], pi = pos[i];
      const T* Di = Dop + (size_t)i * cs;
      for (int t = lane; t < nb2; t += 32) S[t] = blk(Di, co_t, ld, nb, t / nb, t % nb);
      __syncwarp();
      for (int s = 0; s < nf; ++s) {
        const int k = nbr[(size_t)i * nf + s];
        if (k == i || pos[k] > pi) continue;
        // Y = A_ki (k's face blocks towards i)
        for (int t = lane; t < nb2; t += 32) {
          const int r = t / nb, c = t - r * nb;
          T a = T(0);
          for (int s2 = 0; s2 < nf; ++s2)
            if (nbr[(size_t)k * nf + s2] == i) a += blk(O + ((size_t)k * nf + s2) * cs, co_t, ld, nb, r, c);
          Y[t] = a;
        }
        __syncwarp();
        // X = S_k^{-1} Y
        const T* Sk = Sinv + (size_t)k * nb2;
        for (int t = lane; t < nb2; t += 32) {
          const int r = t / nb, c = t - r * nb;
          T a = T(0);
          for (int q = 0; q < nb; ++q) a += Sk[r * nb + q] * Y[q * nb + c];
          X[t] = a;
        }
        __syncwarp();
        // S -= A_i,face s X
        const T* Ob = O + ((size_t)i * nf + s) * cs;
        for (int t = lane; t < nb2; t += 32) {
          const int r = t / nb, c = t - r * nb;
          T a = T(0);
          for (int q = 0; q < nb; ++q) a += blk(Ob, co_t, ld, nb, r, q) * X[q * nb + c];
          S[t] -= a;
        }
        __syncwarp();
      }
      // X = S^{-1}: Gauss-Jordan elimination with partial pivoting (largest
      // |entry| of the column, lowest row on ties)
      for (int t = lane; t < nb2; t += 32) X[t] = (t / nb == t % nb) ? T(1) : T(0);
      __syncwarp();
      for (int cc = 0; cc < nb; ++cc) {
        T bv = T(-1);
        int br = cc;
        for (int r = cc + lane; r < nb; r += 32) {
          const T v = fabs(S[r * nb + cc]);
          if (v > bv) {
            bv = v;
            br = r;
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const T ov = __shfl_xor_sync(0xffffffffu, bv, off);
          const int orr = __shfl_xor_sync(0xffffffffu, br, off);
          if (ov > bv || (ov == bv && orr < br)) {
            bv = ov;
            br = orr;
          }
        }
        if (bv == T(0) && lane == 0) atomicOr(status, ST_SINGULAR);
        if (br != cc)
          for (int t = lane; t < nb; t += 32) {
            const T a = S[cc * nb + t], b = X[cc * nb + t];
            S[cc * nb + t] = S[br * nb + t];
            X[cc * nb + t] = X[br * nb + t];
            S[br * nb + t] = a;
            X[br * nb + t] = b;
          }
        __syncwarp();
        const T piv = S[cc * nb + cc];
        const T inv = piv != T(0) ? T(1) / piv : T(0);
        __syncwarp();
        for (int t = lane; t < nb; t += 32) {
          S[cc * nb + t] *= inv;
          X[cc * nb + t] *= inv;
        }
        __syncwarp();
        for (int r = lane; r < nb; r += 32) {
          if (r == cc) continue;
          const T f = S[r * nb + cc];
          for (int c = cc; c < nb; ++c) S[r * nb + c] -= f * S[cc * nb + c];
          for (int c = 0; c < nb; ++c) X[r * nb + c] -= f * X[cc * nb + c];
        }
        __syncwarp();
      }
      T* So = Sinv + (size_t)i * nb2;
      for (int t = lane; t < nb2; t += 32) So[t] = X[t];
      __syncwarp();
    }
    __syncthreads();
  }
}

// Forward and backward substitution, level by level.  Rows of up to `chunk`
// elements of one level at a time: one thread per (element, row) gathers the
// neighbour products into shared memory, then applies S_i^{-1}.  With
// `resident` the whole vector lives in shared memory during the sweeps.
template <class T>
__global__ void __launch_bounds__(1024) bilu_apply_kernel(const T* __restrict__ Sinv, const T* __restrict__ O,
                                                          size_t cs, int co_t, const int* __restrict__ nbr,
                                                          int nf, const int* __restrict__ pos,
                                                          const int* __restrict__ lptr,
                                                          const int* __restrict__ lel,
                                                          const int* __restrict__ nlev_p, const T* __restrict__ r,
                                                          T* __restrict__ z, int nb, int E, int chunk,
                                                          int resident) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tb = reinterpret_cast<T*>(smem_raw);   // [chunk][nb]
  T* zv = resident ? tb + (size_t)chunk * nb : z;
  const int ld = inv_ld<T>(nb);
  const size_t nb2 = (size_t)nb * nb;
  const int nlev = *nlev_p;
  for (int pass = 0; pass < 2; ++pass) {
    for (int step = 0; step < nlev; ++step) {
      const int lv = pass == 0 ? step : nlev - 1 - step;
      const int beg = lptr[lv], end = lptr[lv + 1];
      for (int c0 = beg; c0 < end; c0 += chunk) {
        const int n = min(chunk, end - c0);
        for (int t = threadIdx.x; t < n * nb; t += blockDim.x) {
          const int el = t / nb, row = t - el * nb, i = lel[c0 + el], pi = pos[i];
          T acc = pass == 0 ? r[(size_t)i * nb + row] : T(0);
          for (int s = 0; s < nf; ++s) {
            const int k = nbr[(size_t)i * nf + s];
            if (k == i || (pass == 0 ? pos[k] > pi : pos[k] < pi)) continue;
            const T* A = O + ((size_t)i * nf + s) * cs;
            const T* zk = zv + (size_t)k * nb;
            T a = T(0);
            for (int c = 0; c < nb; ++c) a += blk(A, co_t, ld, nb, row, c) * zk[c];
            acc -= pass == 0 ? a : -a;
          }
          tb[t] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < n * nb; t += blockDim.x) {
          const int el = t / nb, row = t - el * nb, i = lel[c0 + el];
          const T* Si = Sinv + (size_t)i * nb2 + (size_t)row * nb;
          const T* tv = tb + (size_t)el * nb;
          T acc = T(0);
          for (int c = 0; c < nb; ++c) acc += Si[c] * tv[c];
          if (pass == 0)
            zv[(size_t)i * nb + row] = acc;
          else
            zv[(size_t)i * nb + row] -= acc;
        }
        __syncthreads();
      }
    }
  }
  if (resident)
    for (long t = threadIdx.x; t < (long)E * nb; t += blockDim.x) z[t] = zv[t];
}

size_t smem_budget() {
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)smax;
}

}  // namespace

template <class T>
bool bilu_plan(MG<T>& mg) {
  const Level<T>& L = mg.lv.back();
  const size_t budget = smem_budget(), sz = sizeof(T), row = (size_t)L.nb * sz, E = (size_t)mg.mesh->E;
  const size_t blk3 = 3 * (size_t)L.nb * L.nb * sz;
  if (L.nb > (sizeof(T) == 8 ? 64 : 90) || 2 * blk3 > budget) return false;
  mg.bl_warps = (int)std::min<size_t>(32, budget / blk3);
  const size_t vec = E * row;
  mg.bl_resident = vec + 64 * row <= budget ? 1 : 0;
  const size_t left = budget - (mg.bl_resident ? vec : 0);
  mg.bl_chunk = (int)std::min<size_t>(E, left / row);
  return mg.bl_chunk >= 1;
}

template <class T>
cudaError_t bilu_refresh(MG<T>& mg, cudaStream_t st) {
  const Mesh& M = *mg.mesh;
  const Level<T>& L = mg.lv.back();
  const int E = M.E, nf = 2 * M.d;
  if (mg.bl_kind == DG_ORDER_MDF || mg.h_nlev == 0) {
    if (mg.bl_kind == DG_ORDER_MDF) {
      const long warps = (long)E * nf;
      note_launch();
      bilu_weights_kernel<T><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
          L.Dinv, L.bs, L.inv_t, L.O, L.cs, L.co_t, M.nbr, nf, L.nb, E, mg.bl_c);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      e = cudaMemcpyAsync(mg.h_c.data(), mg.bl_c, sizeof(double) * E * nf, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    }
    const int nl = bilu_order_host(E, nf, mg.h_nbr.data(), mg.h_c.data(), mg.bl_kind, mg.h_order.data(),
                                   mg.h_level.data());
    if (nl < 1) return cudaErrorInvalidValue;
    mg.h_nlev = nl;
    // level schedule: elements by level, in order within a level
    std::vector<int>& ptr = mg.h_ptr;
    std::vector<int>& el = mg.h_el;
    std::vector<int>& pos = mg.h_pos;
    std::fill(ptr.begin(), ptr.end(), 0);
    for (int p = 0; p < E; ++p) {
      pos[mg.h_order[p]] = p;
      ++ptr[mg.h_level[mg.h_order[p]] + 1];
    }
    for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
    std::vector<int> fill(ptr.begin(), ptr.begin() + nl);
    for (int p = 0; p < E; ++p) {
      const int i = mg.h_order[p];
      el[fill[mg.h_level[i]]++] = i;
    }
    mg.h_nlev_buf = nl;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(mg.bl_pos, pos.data(), sizeof(int) * E, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(mg.bl_ptr, ptr.data(), sizeof(int) * (E + 1), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(mg.bl_el, el.data(), sizeof(int) * E, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(mg.bl_nlev, &mg.h_nlev_buf, sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return e;
    // the host arrays are read by the copies above: keep them until they are done
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  const size_t smem = (size_t)mg.bl_warps * 3 * L.nb * L.nb * sizeof(T);
  cudaError_t e = allow_max_smem(bilu_factor_kernel<T>);
  if (e != cudaSuccess) return e;
  note_launch();
  bilu_factor_kernel<T><<<1, 32 * mg.bl_warps, smem, st>>>(L.Dop, L.O, L.cs, L.co_t, M.nbr, nf, mg.bl_pos,
                                                            mg.bl_ptr, mg.bl_el, mg.bl_nlev, mg.Sinv, M.status,
                                                            L.nb);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_bilu_apply(const MG<T>& mg, const T* r, T* z, cudaStream_t st) {
  const Mesh& M = *mg.mesh;
  const Level<T>& L = mg.lv.back();
  const size_t smem = ((size_t)mg.bl_chunk + (mg.bl_resident ? (size_t)M.E : 0)) * L.nb * sizeof(T);
  cudaError_t e = allow_max_smem(bilu_apply_kernel<T>);
  if (e != cudaSuccess) return e;
  note_launch();
  bilu_apply_kernel<T><<<1, 1024, smem, st>>>(mg.Sinv, L.O, L.cs, L.co_t, M.nbr, 2 * M.d, mg.bl_pos, mg.bl_ptr,
                                              mg.bl_el, mg.bl_nlev, r, z, L.nb, M.E, mg.bl_chunk,
                                              mg.bl_resident);
  return cudaGetLastError();
}

template bool bilu_plan<double>(MG<double>&);
template bool bilu_plan<float>(MG<float>&);
template cudaError_t bilu_refresh<double>(MG<double>&, cudaStream_t);
template cudaError_t bilu_refresh<float>(MG<float>&, cudaStream_t);
template cudaError_t launch_bilu_apply<double>(const MG<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_bilu_apply<float>(const MG<float>&, const float*, float*, cudaStream_t);

}  // namespace dgk

extern "C" dg_status dg_bilu_order(int n_elem, int n_faces, const int* nbr, const double* c, int kind, int* order,
                                   int* level, int* n_levels) {
  if (!n_levels) return DG_ERR_INVALID;
  const int nl = dgk::bilu_order_host(n_elem, n_faces, nbr, c, kind, order, level);
  if (nl < 1) return DG_ERR_INVALID;
  *n_levels = nl;
  return DG_OK;
}
