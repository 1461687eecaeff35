// C ABI: residual, JVP, p-multigrid setup/apply and the FGMRES implicit-step
// solve (Sec. 5.1, Sec. 6 with Algorithms 1-2, Sec. 6.1, Sec. 6.3, Sec. 7.4).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <type_traits>

#include "dg_internal.h"

using namespace dgk;

#define CK(...)                                                                    \
  do {                                                                             \
    cudaError_t e__ = (__VA_ARGS__);                                               \
    if (e__ != cudaSuccess) return e__ == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA; \
  } while (0)
#define CKE(...)                        \
  do {                                 \
    cudaError_t e__ = (__VA_ARGS__);   \
    if (e__ != cudaSuccess) return e__; \
  } while (0)

namespace dgk {

// ---------------------------------------------------------------- FD JVP helpers
__global__ void sumsq_partials_kernel(const double* __restrict__ a, long N, int G, double* part) {
  __shared__ double red[256];
  long chunk = (N + G - 1) / G, beg = blockIdx.x * chunk, end = min(N, beg + chunk);
  double s = 0.0;
  for (long n = beg + threadIdx.x; n < end; n += blockDim.x) s += a[n] * a[n];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// scal[0] = ||v||, scal[1] = ||W||, scal[2] = h of eq. DG-mf
__global__ void fd_step_kernel(const double* part, int G, double* scal, int variant, double eps) {
  if (threadIdx.x != 0) return;
  double sv = 0.0, sw = 0.0;
  for (int c = 0; c < G; ++c) sv += part[c];
  for (int c = 0; c < G; ++c) sw += part[1024 + c];
  double nv = sqrt(sv), nw = sqrt(sw);
  scal[0] = nv;
  scal[1] = nw;
  double h;
  if (variant == 0) h = (nw > 0.0) ? eps * sqrt(1.0 + nv) / nw : eps;
  else h = (nv > 0.0) ? eps * sqrt(1.0 + nw) / nv : 0.0;
  scal[2] = h;
}

__global__ void fd_perturb_kernel(long N, const double* W, const double* v, const double* scal, double* out) {
  double h = scal[2];
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x)
    out[n] = W[n] + h * v[n];
}

__global__ void fd_combine_kernel(long N, const double* Rp, const double* RW, const double* v, double sdet,
                                  const double* scal, double* out) {
  double h = scal[2];
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x)
    out[n] = (h > 0.0) ? sdet * v[n] + (Rp[n] - RW[n]) / h : sdet * v[n];
}

static cudaError_t fd_jvp(const Mesh& M, const double* W, const double* RW, double sigma, const double* v,
                          double* out, int variant, cudaStream_t st) {
  long N = (long)M.E * M.nb;
  int G = (int)std::min<long>(1024, std::max<long>(1, (N + 4095) / 4096));
  note_launch();
  sumsq_partials_kernel<<<G, 256, 0, st>>>(v, N, G, M.partials);
  note_launch();
  sumsq_partials_kernel<<<G, 256, 0, st>>>(W, N, G, M.partials + 1024);
  note_launch();
  fd_step_kernel<<<1, 32, 0, st>>>(M.partials, G, M.scal, variant, 1e-7);
  int gr = (int)std::min<long>((N + 255) / 256, 4096);
  note_launch();
  fd_perturb_kernel<<<gr, 256, 0, st>>>(N, W, v, M.scal, M.t64.fd_w);
  CKE(cudaGetLastError());
  CKE(launch_residual<double>(M, M.t64.fd_w, nullptr, nullptr, 0.0, false, M.t64.fd_r, st));
  note_launch();
  fd_combine_kernel<<<gr, 256, 0, st>>>(N, M.t64.fd_r, RW, v, sigma * M.detJ, M.scal, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- multigrid
template <class T>
cudaError_t MG<T>::op(int l, const T* x, T* y, cudaStream_t st) {
  if (l == 0) return launch_residual<T>(*mesh, W, x, nullptr, sigma, true, y, st, Pv, Pf);
  Level<T>& L = lv[l];
  if (L.Dop16)   // BF16 storage (FP32 handles only)
    return launch_bsr_bf16(L.Dop16, L.O16, mesh->face_nbr(), mesh->nfaces(), reinterpret_cast<const float*>(x),
                           reinterpret_cast<float*>(y), L.nb, mesh->E, st);
  return launch_bsr<T>(L.Dop, L.O, L.cs, L.co_t, mesh->face_nbr(), mesh->nfaces(), x, y, L.nb, mesh->E, st);
}

// z = D_l^{-1} r with the level's stored inverses (block Jacobi, Sec. 6.3).
template <class T>
static cudaError_t bj_apply(const Level<T>& L, const T* r, T* z, int E, cudaStream_t st) {
  if (L.Dinv16)
    return launch_block_apply_bf16(L.Dinv16, reinterpret_cast<const float*>(r), reinterpret_cast<float*>(z), L.nb,
                                   E, st);
  return launch_block_apply<T>(L.Dinv, L.bs, L.inv_t, r, z, L.nb, E, st);
}

// SMOOTH / SOLVE: nu iterations of GMRES right-preconditioned by block Jacobi
// (block ILU(0) on the coarsest level when asked: Table MGSettings), from the
// current x (Algorithm 2), no restart.
template <class T>
cudaError_t MG<T>::smooth(int l, const T* b, T* x, int nu, cudaStream_t st) {
  Level<T>& L = lv[l];
  Krylov<T>& K = L.kr;
  if constexpr (std::is_same<T, float>::value) {
    // inherited FP32/BF16 coarse levels: the whole call in one persistent launch
    const bool ilu = bilu && l == (int)lv.size() - 1;
    if (l >= 1 && L.coop.ok && !ilu && (L.Dinv16 || (L.inv_t && L.co_t))) {
      if (nu == 0) return cudaSuccess;
      return launch_coop_smoother(L.coop, L.Dinv, L.Dop, L.O, L.Dinv16, L.Dop16, L.O16, mesh->face_nbr(),
                                  mesh->nfaces(), b, x, nu, K, L.cpart, L.cbar, mesh->status, coop_extra, L.nb,
                                  mesh->E, st);
    }
  }
  CKE(op(l, x, L.r, st));
  CKE(launch_axpby<T>(L.N, 1.0, b, -1.0, L.r, st));           // r = b - A x
  CKE(K.start(L.r, st));
  const bool ilu = bilu && l == (int)lv.size() - 1;   // block ILU(0) on the coarsest level
  for (int j = 0; j < nu; ++j) {
    if (ilu)
      CKE(launch_bilu_apply<T>(*this, K.Vj(j), K.Zj(j), st));
    else
      CKE(bj_apply<T>(L, K.Vj(j), K.Zj(j), mesh->E, st));
    CKE(op(l, K.Zj(j), K.w, st));
    CKE(K.arnoldi(j, st));
  }
  return K.update(nu, x, st);
}

// MG_V(l, b_l, x_l) of Algorithm 2 on lv[l].b / lv[l].x (x updated in place).
template <class T>
cudaError_t MG<T>::mg_v(int l, cudaStream_t st) {
  const int Lc = (int)lv.size() - 1;
  Level<T>& L = lv[l];
  if (l == Lc) return smooth(l, L.b, L.x, nu_coarse, st);
  CKE(smooth(l, L.b, L.x, L.nu_pre, st));
  CKE(op(l, L.x, L.t, st));
  CKE(launch_axpby<T>(L.N, 1.0, L.b, -1.0, L.t, st));         // r_l = b_l - A_l x_l
  Level<T>& C = lv[l + 1];
  CKE(launch_restrict<T>(L.t, L.nm, C.b, C.nm, (long)mesh->E * mesh->m, st));
  CKE(cudaMemsetAsync(C.x, 0, sizeof(T) * C.N, st));
  CKE(mg_v(l + 1, st));
  CKE(launch_prolong<T>(C.x, C.nm, L.x, L.nm, (long)mesh->E * mesh->m, true, st));
  return smooth(l, L.b, L.x, L.nu_post, st);
}

// One preconditioner application z = P^{-1} r.
template <class T>
cudaError_t MG<T>::apply(const T* r, T* z, cudaStream_t st) {
  const int Lc = (int)lv.size() - 1;
  const long nev = (long)mesh->E * mesh->m;
  if (cycle == DG_CYCLE_BJ)
    return bj_apply<T>(lv[0], r, z, mesh->E, st);
  // (copies by kernel: the application is also captured into conditional graph
  // bodies, where kernels and memsets are the node types used)
  if (cycle == DG_CYCLE_V) {
    CKE(launch_axpby<T>(lv[0].N, 1.0, r, 0.0, lv[0].b, st));
    CKE(cudaMemsetAsync(lv[0].x, 0, sizeof(T) * lv[0].N, st));
    CKE(mg_v(0, st));
    return launch_axpby<T>(lv[0].N, 1.0, lv[0].x, 0.0, z, st);
  }
  // MG_full (Algorithm 1): b_l = I_0^l b_0 on every level, SOLVE on the
  // coarsest, then for l = L-1..0: x~_l = I_{l+1}^l x_{l+1}, x_l = MG_V(l, b_l, x~_l)
  CKE(launch_axpby<T>(lv[0].N, 1.0, r, 0.0, lv[0].b, st));
  for (int l = 1; l <= Lc; ++l) CKE(launch_restrict<T>(r, lv[0].nm, lv[l].b, lv[l].nm, nev, st));
  CKE(cudaMemsetAsync(lv[Lc].x, 0, sizeof(T) * lv[Lc].N, st));
  CKE(smooth(Lc, lv[Lc].b, lv[Lc].x, nu_coarse, st));
  for (int l = Lc - 1; l >= 0; --l) {
    CKE(launch_prolong<T>(lv[l + 1].x, lv[l + 1].nm, lv[l].x, lv[l].nm, nev, false, st));
    CKE(mg_v(l, st));
  }
  return launch_axpby<T>(lv[0].N, 1.0, lv[0].x, 0.0, z, st);
}

template struct MG<double>;
template struct MG<float>;

static cudaError_t dalloc(std::vector<void*>& list, void** p, size_t bytes, size_t* counter) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e == cudaSuccess) {
    list.push_back(*p);
    if (counter) *counter += bytes;
  }
  return e;
}

template <class T>
static dg_status alloc_mg(dg_pmg h, MG<T>& mg) {
  const Mesh& M = h->mesh->m;
  const dg_pmg_opts& o = h->opts;
  mg.mesh = &M;
  mg.nu_coarse = o.nu_coarse;
  const char* extra = getenv("DG_TEST_COOP_BARRIER_EXTRA");   // test hook: a barrier that is never met
  mg.coop_extra = extra ? std::max(0, atoi(extra)) : 0;
  mg.cycle = o.cycle;
  const int nl = o.cycle == DG_CYCLE_BJ ? 1 : o.n_levels;
  mg.lv.resize(nl);
  const long N0 = (long)M.E * M.nb;
  CK(dalloc(mg.allocs, (void**)&mg.W, sizeof(T) * N0, &h->vector_bytes));
  for (int l = 0; l < nl; ++l) {
    Level<T>& L = mg.lv[l];
    L.p = o.p_level[l];
    long c = 1;  // n_m = C(p + d, d)
    if (M.desc.space == DG_SPACE_Q)
      for (int i = 1; i <= M.d; ++i) c *= L.p + 1;
    else
      for (int i = 1; i <= M.d; ++i) c = c * (L.p + i) / i;
    L.nm = (int)c;
    L.nb = M.m * L.nm;
    L.N = (long)M.E * L.nb;
    L.nu_pre = o.nu_pre[l];
    L.nu_post = o.nu_post[l];
    size_t nbl = (size_t)M.E * L.nb * L.nb;
    L.bs = (size_t)L.nb * inv_ld<T>(L.nb);
    CK(dalloc(mg.allocs, (void**)&L.Dinv, sizeof(T) * (size_t)M.E * L.bs, &h->block_bytes));
    if (l >= 1) {
      // coarse blocks column-major when the FP32 neighbour blocks come from
      // probe_nbr_kernel (decided here once: the captured graph relies on it)
      // (the column-major mat-vec runs one thread per block and 16 bytes of rows: at most 256 per element)
      const int tpb1 = (1 + 2 * M.d) * (inv_ld<T>(mg.lv[1].nb) / (int)(16 / sizeof(T)));
      L.co_t = M.kind == DG_MESH_STRUCTURED && std::is_same<T, float>::value && tpb1 <= 256 &&
                       probe_nbr_colmajor_ok(M, mg.lv[1].nm) ? 1 : 0;
      L.cs = L.co_t ? L.bs : (size_t)L.nb * L.nb;
      (void)nbl;
      CK(dalloc(mg.allocs, (void**)&L.Dop, sizeof(T) * (size_t)M.E * L.cs, &h->block_bytes));
      CK(dalloc(mg.allocs, (void**)&L.O, sizeof(T) * (size_t)M.E * M.nfaces() * L.cs, &h->block_bytes));
      CK(cudaMemset(L.Dop, 0, sizeof(T) * (size_t)M.E * L.cs));   // padding rows stay zero
      CK(cudaMemset(L.O, 0, sizeof(T) * (size_t)M.E * M.nfaces() * L.cs));
    }
    if (o.block_storage == DG_STORE_BF16) {   // mixed precision only (check_opts)
      const size_t b16 = (size_t)L.nb * ld_bf16(L.nb) * sizeof(unsigned short);
      CK(dalloc(mg.allocs, (void**)&L.Dinv16, b16 * M.E, &h->block_bytes));
      if (l >= 1) {
        CK(dalloc(mg.allocs, (void**)&L.Dop16, b16 * M.E, &h->block_bytes));
        CK(dalloc(mg.allocs, (void**)&L.O16, b16 * M.E * M.nfaces(), &h->block_bytes));
      }
    }
    for (T** v : {&L.x, &L.b, &L.r, &L.t}) CK(dalloc(mg.allocs, (void**)v, sizeof(T) * L.N, &h->vector_bytes));
    int nmax = (l == nl - 1) ? std::max(1, o.nu_coarse) : std::max(std::max(L.nu_pre, L.nu_post), 1);
    if (o.cycle != DG_CYCLE_BJ) {
      CK(L.kr.alloc(L.N, nmax));
      h->vector_bytes += L.kr.bytes();
    }
    // persistent smoother of an inherited FP32 level (column-major or BF16
    // blocks, face-neighbour graph of the structured mesh); DG_PMG_NO_COOP=1
    // keeps the launch-per-operation smoother
    const char* nco = getenv("DG_PMG_NO_COOP");
    const bool bf16 = o.block_storage == DG_STORE_BF16;
    if (std::is_same<T, float>::value && l >= 1 && o.cycle != DG_CYCLE_BJ && M.kind == DG_MESH_STRUCTURED &&
        (L.co_t || bf16) && !(nco && nco[0] == '1') &&
        !(o.coarse_precond == DG_COARSE_BILU && l == nl - 1)) {
      CK(plan_coop_smoother(bf16 ? 1 : 0, L.nb, M.nfaces(), M.E, nmax, &L.coop));
      if (L.coop.ok) {
        L.coop.nu_max = nmax;
        CK(dalloc(mg.allocs, (void**)&L.cpart, sizeof(double) * (size_t)(L.coop.grid + 1) * (2 * (nmax + 1) + 1),
                  &h->vector_bytes));
        CK(dalloc(mg.allocs, (void**)&L.cbar, sizeof(unsigned) * COOP_BAR_WORDS, &h->vector_bytes));
      }
    }
  }
  // primal traces of the fine JVP's linearisation point (FP32 smoother JVPs);
  // DG_PMG_NO_PRIMAL_CACHE=1 makes every JVP interpolate W itself
  const char* npc = getenv("DG_PMG_NO_PRIMAL_CACHE");
  if (M.kind == DG_MESH_STRUCTURED && std::is_same<T, float>::value && !(npc && npc[0] == '1') &&
      o.cycle != DG_CYCLE_BJ) {
    size_t nf = 0, nv = primal_cache_sizes(M, &nf);
    CK(dalloc(mg.allocs, (void**)&mg.Pv, sizeof(T) * nv, &h->vector_bytes));
    CK(dalloc(mg.allocs, (void**)&mg.Pf, sizeof(T) * nf, &h->vector_bytes));
  }
  if (o.coarse_precond == DG_COARSE_BILU) {
    const Level<T>& C = mg.lv.back();
    const int nf = 2 * M.d;
    mg.bilu = 1;
    mg.bl_kind = o.coarse_order;
    if (!bilu_plan(mg)) return DG_ERR_INVALID;
    CK(dalloc(mg.allocs, (void**)&mg.Sinv, sizeof(T) * (size_t)M.E * C.nb * C.nb, &h->block_bytes));
    CK(dalloc(mg.allocs, (void**)&mg.bl_pos, sizeof(int) * M.E, &h->vector_bytes));
    CK(dalloc(mg.allocs, (void**)&mg.bl_ptr, sizeof(int) * (M.E + 1), &h->vector_bytes));
    CK(dalloc(mg.allocs, (void**)&mg.bl_el, sizeof(int) * M.E, &h->vector_bytes));
    CK(dalloc(mg.allocs, (void**)&mg.bl_nlev, sizeof(int), &h->vector_bytes));
    CK(dalloc(mg.allocs, (void**)&mg.bl_c, sizeof(double) * M.E * nf, &h->vector_bytes));
    mg.h_nbr.resize((size_t)M.E * nf);
    CK(cudaMemcpy(mg.h_nbr.data(), M.nbr, sizeof(int) * M.E * nf, cudaMemcpyDeviceToHost));
    mg.h_c.assign((size_t)M.E * nf, 0.0);
    mg.h_order.assign(M.E, 0);
    mg.h_level.assign(M.E, 0);
    mg.h_pos.assign(M.E, 0);
    mg.h_el.assign(M.E, 0);
    mg.h_ptr.assign(M.E + 1, 0);
    mg.h_nlev = 0;
  }
  // probing caches live in global memory when they exceed shared memory
  bool fits = true;
  size_t tot = M.kind == DG_MESH_STRUCTURED ? probe_scratch_elems<T>(M, nl > 1 ? mg.lv[1].nm : 0, &fits) : 0;
  if (!fits) {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    mg.scratch_elems = tot * (size_t)std::min(M.E, 2 * nsm);
    CK(dalloc(mg.allocs, (void**)&mg.scratch, sizeof(T) * mg.scratch_elems, &h->block_bytes));
  }
  return DG_OK;
}

// Preconditioner at state W and shift sigma into the allocated handle: fine
// diagonal blocks (+ neighbour blocks at the first coarse order) by probing,
// coarse blocks by truncation (inheritance), block inverses.  Asynchronous.
template <class T>
static dg_status compute_mg(dg_pmg h, MG<T>& mg, const double* W64, cudaStream_t st) {
  const Mesh& M = h->mesh->m;
  const int nl = (int)mg.lv.size();
  const long N0 = (long)M.E * M.nb;
  mg.sigma = (T)h->sigma;
  if (std::is_same<T, double>::value)
    CK(cudaMemcpyAsync(mg.W, W64, sizeof(double) * N0, cudaMemcpyDeviceToDevice, st));
  else
    CK(launch_convert<double, float>(N0, W64, (float*)mg.W, st));
  if (mg.Pv) CK(launch_primal_cache(M, (const float*)mg.W, (float*)mg.Pv, (float*)mg.Pf, st));
  if (M.kind == DG_MESH_TRI)   // coloured JVP probing, seeds and products in level 0's work vectors
    CK(launch_probe_blocks_tri<T>(M, mg.W, (T)h->sigma, mg.lv[0].Dinv, mg.lv[0].bs, nl > 1 ? mg.lv[1].O : nullptr,
                                  nl > 1 ? mg.lv[1].nm : 0, mg.lv[0].r, mg.lv[0].t, st));
  else
    CK(launch_probe_blocks<T>(M, mg.W, (T)h->sigma, mg.lv[0].Dinv, mg.lv[0].bs, nl > 1 ? mg.lv[1].O : nullptr,
                              nl > 1 ? mg.lv[1].nm : 0, nl > 1 ? mg.lv[1].co_t : 0, mg.scratch, mg.scratch_elems,
                              st));
  const Level<T>& F = mg.lv[0];
  for (int l = 1; l < nl; ++l) {
    Level<T>& L = mg.lv[l];
    // inherited diagonal blocks: for the operator (layout of the level) and,
    // row-major, as the input of the inverse
    CK(launch_truncate_blocks<T>(F.Dinv, F.nm, F.bs, 0, L.Dop, L.nm, L.cs, L.co_t, M.m, M.E, st));
    CK(launch_truncate_blocks<T>(F.Dinv, F.nm, F.bs, 0, L.Dinv, L.nm, L.bs, 0, M.m, M.E, st));
    if (l >= 2)
      CK(launch_truncate_blocks<T>(mg.lv[1].O, mg.lv[1].nm, mg.lv[1].cs, mg.lv[1].co_t, L.O, L.nm, L.cs, L.co_t,
                                   M.m, (long)M.E * M.nfaces(), st));
  }
  for (int l = 0; l < nl; ++l)
    CK(launch_block_inverse<T>(mg.lv[l].Dinv, mg.lv[l].nb, mg.lv[l].bs, M.E, M.status, &mg.lv[l].inv_t, st));
  for (int l = 0; l < nl; ++l) {   // BF16 copies the smoothers stream (round to nearest)
    Level<T>& L = mg.lv[l];
    if (!L.Dinv16) continue;
    CK(launch_to_bf16(reinterpret_cast<const float*>(L.Dinv), L.bs, L.inv_t, L.Dinv16, L.nb, M.E, st));
    if (l >= 1) {
      CK(launch_to_bf16(reinterpret_cast<const float*>(L.Dop), L.cs, L.co_t, L.Dop16, L.nb, M.E, st));
      CK(launch_to_bf16(reinterpret_cast<const float*>(L.O), L.cs, L.co_t, L.O16, L.nb, (long)M.E * M.nfaces(),
                        st));
    }
  }
  if (mg.bilu) CK(bilu_refresh<T>(mg, st));
  return DG_OK;
}

static void free_list(std::vector<void*>& l) {
  for (void* p : l) cudaFree(p);
  l.clear();
}

template <class T>
static void free_mg(MG<T>& mg) {
  for (auto& L : mg.lv) L.kr.release();
  free_list(mg.allocs);
  mg.lv.clear();
}

}  // namespace dgk

// ====================================================================== ABI
extern "C" dg_status dg_residual(dg_mesh mesh, const double* W, const double* S, double* R, void* stream) {
  if (!mesh || !W || !R || R == W || (S && S == R)) return DG_ERR_INVALID;
  CK(launch_residual<double>(mesh->m, W, nullptr, S, 0.0, false, R, (cudaStream_t)stream));
  return DG_OK;
}

extern "C" dg_status dg_jvp(dg_mesh mesh, const double* W, const double* R_W, double sigma, const double* v,
                            double* Kv, int mode, void* stream) {
  if (!mesh || !W || !v || !Kv || Kv == W || Kv == v) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == DG_JVP_EXACT) {
    CK(launch_residual<double>(mesh->m, W, v, nullptr, sigma, true, Kv, st));
    return DG_OK;
  }
  if (mode == DG_JVP_EXACT_FP32) {   // the mixed-precision smoother's operator
    const Mesh& M = mesh->m;
    const long N = (long)M.E * M.nb;
    CK(launch_convert<double, float>(N, W, M.t32.fd_w, st));
    CK(launch_convert<double, float>(N, v, M.t32.fd_r, st));
    CK(launch_residual<float>(M, M.t32.fd_w, M.t32.fd_r, nullptr, (float)sigma, true, M.t32.fd_o, st));
    CK(launch_convert<float, double>(N, M.t32.fd_o, Kv, st));
    return DG_OK;
  }
  if (mode != DG_JVP_FD && mode != DG_JVP_FD_SCALED) return DG_ERR_INVALID;
  if (!R_W || R_W == Kv || mesh->m.kind != DG_MESH_STRUCTURED) return DG_ERR_INVALID;
  CK(fd_jvp(mesh->m, W, R_W, sigma, v, Kv, mode == DG_JVP_FD ? 0 : 1, st));
  return DG_OK;
}

// Capture one preconditioner application (every level, every smoother
// iteration: a few thousand small launches) as a CUDA graph on fixed staging
// buffers.  The graph reads the handle's blocks and state through pointers, so
// a refresh at the same shift keeps it; the shift itself is a by-value kernel
// argument, so a refresh at another shift captures it again.
// DG_PMG_NO_GRAPH=1 disables it.
static dg_status capture_apply_graph(dg_pmg h) {
  const char* env = getenv("DG_PMG_NO_GRAPH");
  if (env && env[0] == '1') return DG_OK;
  const long N0 = (long)h->mesh->m.E * h->mesh->m.nb;
  if (!h->cap_stream) {
    if (h->precision == DG_PREC_FP64) {
      if (dalloc(h->allocs, (void**)&h->r64, sizeof(double) * N0, &h->vector_bytes) != cudaSuccess ||
          dalloc(h->allocs, (void**)&h->z64, sizeof(double) * N0, &h->vector_bytes) != cudaSuccess)
        return DG_ERR_OOM;
    }
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  }
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph_exec = nullptr;
  h->graph = nullptr;
  h->graph_sigma = h->sigma;
  unsigned long long l0 = __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED);
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
  cudaError_t e = h->precision == DG_PREC_FP64 ? h->mg64.apply(h->r64, h->z64, h->cap_stream)
                                               : h->mg32.apply(h->r32, h->z32, h->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return DG_ERR_CUDA;
  }
  h->graph = g;
  h->graph_kernels = __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED) - l0;
  __atomic_fetch_sub(&launch_counter(), h->graph_kernels, __ATOMIC_RELAXED);   // captured, not run
  CK(cudaGraphInstantiate(&h->graph_exec, h->graph, 0));
  return DG_OK;
}

static dg_status check_opts(const dg_mesh_s* mesh, const dg_pmg_opts* o) {
  if (o->cycle != DG_CYCLE_FMG && o->cycle != DG_CYCLE_V && o->cycle != DG_CYCLE_BJ) return DG_ERR_INVALID;
  if (o->precision != DG_PREC_FP64 && o->precision != DG_PREC_MIXED) return DG_ERR_INVALID;
  if (o->fgmres_restart < 0 || o->fgmres_restart > 64) return DG_ERR_INVALID;
  if (o->coarse_precond != DG_COARSE_BJ && o->coarse_precond != DG_COARSE_BILU) return DG_ERR_INVALID;
  if (o->block_storage != DG_STORE_NATIVE && o->block_storage != DG_STORE_BF16) return DG_ERR_INVALID;
  if (o->block_storage == DG_STORE_BF16) {
    // FP32 handles only; the BSR kernel runs a thread per block and 8 rows of every element
    if (o->precision != DG_PREC_MIXED) return DG_ERR_INVALID;
    const int nl = o->cycle == DG_CYCLE_BJ ? 1 : o->n_levels;
    for (int l = 0; l < nl && l < 8; ++l) {
      const int p = o->cycle == DG_CYCLE_BJ ? mesh->m.p : o->p_level[l];
      long c = 1;
      if (mesh->m.desc.space == DG_SPACE_Q)
        for (int i = 1; i <= mesh->m.d; ++i) c *= p + 1;
      else
        for (int i = 1; i <= mesh->m.d; ++i) c = c * (p + i) / i;
      const int nb = mesh->m.m * (int)c;
      if (ld_bf16(nb) / 8 > 256 || (l >= 1 && (1 + mesh->m.nfaces()) * (ld_bf16(nb) / 8) > 256))
        return DG_ERR_INVALID;
    }
  }
  if (o->coarse_precond == DG_COARSE_BILU) {
    // neighbour blocks exist from level 1; the pivot-block form of ILU(0)
    // needs a face graph without triangles (no periodic direction of 3)
    if (o->cycle == DG_CYCLE_BJ || o->n_levels < 2) return DG_ERR_INVALID;
    if (o->coarse_order < DG_ORDER_MDF || o->coarse_order > DG_ORDER_COLOUR) return DG_ERR_INVALID;
    if (mesh->m.kind != DG_MESH_STRUCTURED) return DG_ERR_INVALID;
    for (int k = 0; k < mesh->m.d; ++k)
      if (mesh->m.desc.n[k] == 3) return DG_ERR_INVALID;
  }
  if (o->cycle == DG_CYCLE_BJ) return o->p_level[0] == mesh->m.p || o->n_levels == 0 ? DG_OK : DG_ERR_INVALID;
  if (o->n_levels < 1 || o->n_levels > 8) return DG_ERR_INVALID;
  if (o->p_level[0] != mesh->m.p) return DG_ERR_INVALID;
  for (int l = 1; l < o->n_levels; ++l)
    if (o->p_level[l] < 0 || o->p_level[l] >= o->p_level[l - 1]) return DG_ERR_INVALID;
  if (o->nu_coarse < 1 || o->nu_coarse > 64) return DG_ERR_INVALID;
  for (int l = 0; l + 1 < o->n_levels; ++l)
    if (o->nu_pre[l] < 0 || o->nu_post[l] < 0 || o->nu_pre[l] > 64 || o->nu_post[l] > 64) return DG_ERR_INVALID;
  return DG_OK;
}

extern "C" dg_status dg_pmg_destroy(dg_pmg h) {
  if (!h) return DG_ERR_INVALID;
  if (h->fgm_exec) cudaGraphExecDestroy(h->fgm_exec);
  if (h->fgm_graph) cudaGraphDestroy(h->fgm_graph);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  free_mg(h->mg64);
  free_mg(h->mg32);
  h->outer.release();
  free_list(h->allocs);
  delete h;
  return DG_OK;
}

extern "C" dg_status dg_pmg_setup(dg_mesh mesh, const double* W, double sigma, const dg_pmg_opts* opts,
                                  void* stream, dg_pmg* out) {
  if (!out) return DG_ERR_INVALID;
  *out = nullptr;
  if (!mesh || !W || !opts || !(sigma >= 0.0)) return DG_ERR_INVALID;
  dg_status s = check_opts(mesh, opts);
  if (s != DG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  dg_pmg h = new dg_pmg_s();
  h->mesh = mesh;
  h->opts = *opts;
  if (h->opts.cycle == DG_CYCLE_BJ) {
    h->opts.n_levels = 1;
    h->opts.p_level[0] = mesh->m.p;
  }
  h->sigma = sigma;
  h->precision = opts->precision;
  CK(cudaMemsetAsync(mesh->m.status, 0, sizeof(int), st));
  if (h->precision == DG_PREC_FP64) {
    s = alloc_mg<double>(h, h->mg64);
    if (s == DG_OK) s = compute_mg<double>(h, h->mg64, W, st);
  } else {
    s = alloc_mg<float>(h, h->mg32);
    if (s == DG_OK) s = compute_mg<float>(h, h->mg32, W, st);
  }
  const long N0 = (long)mesh->m.E * mesh->m.nb;
  if (s == DG_OK && h->precision == DG_PREC_MIXED) {
    if (dalloc(h->allocs, (void**)&h->r32, sizeof(float) * N0, &h->vector_bytes) != cudaSuccess ||
        dalloc(h->allocs, (void**)&h->z32, sizeof(float) * N0, &h->vector_bytes) != cudaSuccess)
      s = DG_ERR_OOM;
  }
  if (s == DG_OK) {
    h->outer_restart = opts->fgmres_restart > 0 ? opts->fgmres_restart : 30;
    if (h->outer.alloc(N0, h->outer_restart) != cudaSuccess ||
        dalloc(h->allocs, (void**)&h->tmp64, sizeof(double) * N0 * 2, &h->vector_bytes) != cudaSuccess)
      s = DG_ERR_OOM;
    else
      h->vector_bytes += h->outer.bytes();
  }
  if (s == DG_OK) {
    int hs = 0;
    if (cudaMemcpyAsync(&hs, mesh->m.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = DG_ERR_CUDA;
    else if (hs & ST_TIMEOUT)
      s = DG_ERR_TIMEOUT;
    else if (hs & ST_SINGULAR)
      s = DG_ERR_BREAKDOWN;
    else if (hs & ST_NONPHYSICAL)
      s = DG_ERR_NONPHYSICAL;
  }
  if (s == DG_OK) s = capture_apply_graph(h);
  if (s != DG_OK) {
    dg_pmg_destroy(h);
    return s;
  }
  *out = h;
  return DG_OK;
}

extern "C" dg_status dg_pmg_refresh(dg_pmg h, const double* W, double sigma, void* stream) {
  if (!h || !W || !(sigma >= 0.0)) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  h->sigma = sigma;
  dg_status s = h->precision == DG_PREC_FP64 ? compute_mg<double>(h, h->mg64, W, st)
                                             : compute_mg<float>(h, h->mg32, W, st);
  if (s == DG_OK && h->graph_exec && h->graph_sigma != sigma) s = capture_apply_graph(h);
  return s;
}

static dg_status pmg_apply_impl(dg_pmg h, const double* r, double* z, cudaStream_t st) {
  const long N0 = (long)h->mesh->m.E * h->mesh->m.nb;
  if (h->graph_exec) {
    // replay the captured application between fixed staging buffers
    if (h->precision == DG_PREC_FP64) {
      CK(cudaMemcpyAsync(h->r64, r, sizeof(double) * N0, cudaMemcpyDeviceToDevice, st));
      CK(cudaGraphLaunch(h->graph_exec, st));
      CK(cudaMemcpyAsync(z, h->z64, sizeof(double) * N0, cudaMemcpyDeviceToDevice, st));
    } else {
      CK(launch_convert<double, float>(N0, r, h->r32, st));
      CK(cudaGraphLaunch(h->graph_exec, st));
      CK(launch_convert<float, double>(N0, h->z32, z, st));
    }
    __atomic_fetch_add(&launch_counter(), h->graph_kernels, __ATOMIC_RELAXED);
    return DG_OK;
  }
  if (h->precision == DG_PREC_FP64) {
    CK(h->mg64.apply(r, z, st));
  } else {
    CK(launch_convert<double, float>(N0, r, h->r32, st));
    CK(h->mg32.apply(h->r32, h->z32, st));
    CK(launch_convert<float, double>(N0, h->z32, z, st));
  }
  return DG_OK;
}

extern "C" dg_status dg_pmg_apply(dg_pmg h, const double* r, double* z, void* stream) {
  if (!h || !r || !z || r == z) return DG_ERR_INVALID;
  return pmg_apply_impl(h, r, z, (cudaStream_t)stream);
}

extern "C" dg_status dg_pmg_operator(dg_pmg h, int level, const double* x, double* y, void* stream) {
  if (!h || !x || !y || x == y) return DG_ERR_INVALID;
  const bool f64 = h->precision == DG_PREC_FP64;
  const int nl = (int)(f64 ? h->mg64.lv.size() : h->mg32.lv.size());
  if (level < 0 || level >= nl) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (f64) {
    CK(h->mg64.op(level, x, y, st));
    return DG_OK;
  }
  const long N = h->mg32.lv[level].N;   // <= the fine level's size of the staging buffers
  CK(launch_convert<double, float>(N, x, h->r32, st));
  CK(h->mg32.op(level, h->r32, h->z32, st));
  CK(launch_convert<float, double>(N, h->z32, y, st));
  return DG_OK;
}

namespace dgk {
// deterministic non-zero input for kernel timing: x[i] in [-1e-3, 1e-3)
template <class T>
__global__ void fill_pattern_kernel(T* x, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[i] = (T)(1e-3 * ((double)((i * 7919) % 1000) - 500.0) / 500.0);
}

template <class T>
static dg_status time_kernel(MG<T>& mg, const Mesh& M, int kernel, int level, int reps, float* ms,
                             cudaStream_t st) {
  Level<T>& L = mg.lv[level];
  const int grid = (int)std::min<long>((L.N + 255) / 256, 4096);
  note_launch();
  fill_pattern_kernel<T><<<grid, 256, 0, st>>>(L.r, L.N);
  note_launch();
  fill_pattern_kernel<T><<<grid, 256, 0, st>>>(L.b, L.N);
  CK(cudaMemsetAsync(L.x, 0, sizeof(T) * L.N, st));
  const int nu = level == (int)mg.lv.size() - 1 ? mg.nu_coarse : std::max(1, L.nu_pre);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    switch (kernel) {
      case DG_KT_FACE_JVP:
        e = launch_residual<T>(M, mg.W, L.r, nullptr, mg.sigma, true, L.t, st, mg.Pv, mg.Pf, 1);
        break;
      case DG_KT_VOLUME_JVP:
        e = launch_residual<T>(M, mg.W, L.r, nullptr, mg.sigma, true, L.t, st, mg.Pv, mg.Pf, 2);
        break;
      case DG_KT_BLOCK_JACOBI:
        e = bj_apply<T>(L, L.r, L.t, M.E, st);
        break;
      case DG_KT_OPERATOR:
        e = mg.op(level, L.r, L.t, st);
        break;
      default:
        e = mg.smooth(level, L.b, L.x, nu, st);
        break;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(e);
  *ms = t / (float)reps;
  return DG_OK;
}
}  // namespace dgk

extern "C" dg_status dg_pmg_kernel_time(dg_pmg h, int kernel, int level, int reps, float* ms, void* stream) {
  if (!h || !ms || reps < 1 || kernel < DG_KT_FACE_JVP || kernel > DG_KT_SMOOTH) return DG_ERR_INVALID;
  const Mesh& M = h->mesh->m;
  const bool f64 = h->precision == DG_PREC_FP64;
  const int nl = (int)(f64 ? h->mg64.lv.size() : h->mg32.lv.size());
  if (level < 0 || level >= nl || M.kind != DG_MESH_STRUCTURED) return DG_ERR_INVALID;
  if ((kernel == DG_KT_FACE_JVP || kernel == DG_KT_VOLUME_JVP) && level != 0) return DG_ERR_INVALID;
  if (kernel == DG_KT_SMOOTH && (nl == 1 && h->opts.cycle == DG_CYCLE_BJ)) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  return f64 ? time_kernel<double>(h->mg64, M, kernel, level, reps, ms, st)
             : time_kernel<float>(h->mg32, M, kernel, level, reps, ms, st);
}

extern "C" dg_status dg_pmg_bilu_order(dg_pmg h, int* order, int* n_levels, void* stream) {
  if (!h || !n_levels) return DG_ERR_INVALID;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DG_ERR_CUDA;
  const bool f64 = h->precision == DG_PREC_FP64;
  const int on = f64 ? h->mg64.bilu : h->mg32.bilu;
  if (!on) return DG_ERR_INVALID;
  const std::vector<int>& o = f64 ? h->mg64.h_order : h->mg32.h_order;
  *n_levels = f64 ? h->mg64.h_nlev : h->mg32.h_nlev;
  if (order) std::copy(o.begin(), o.end(), order);
  return DG_OK;
}

extern "C" dg_status dg_pmg_bytes(dg_pmg h, size_t* block_bytes, size_t* vector_bytes) {
  if (!h) return DG_ERR_INVALID;
  if (block_bytes) *block_bytes = h->block_bytes;
  if (vector_bytes) *vector_bytes = h->vector_bytes;
  return DG_OK;
}

// Row-major packed copy of a level's blocks (any storage layout).
template <class T>
static dg_status export_level(const MG<T>& mg, const Mesh& M, T* W, double sigma, int level, int which, T* out,
                              size_t out_bytes, cudaStream_t st) {
  const Level<T>& L = mg.lv[level];
  const int nb = L.nb;
  const size_t nblk = which == DG_BLOCKS_NEIGHBOUR ? (size_t)M.E * M.nfaces() : (size_t)M.E;
  if (out_bytes < nblk * nb * nb * sizeof(T)) return DG_ERR_INVALID;
  if (which == DG_BLOCKS_DIAG_INV) {
    if (L.Dinv16)
      CK(launch_unpack_bf16(L.Dinv16, reinterpret_cast<float*>(out), nb, (long)nblk, st));
    else
      CK(launch_unpack_inverse<T>(L.Dinv, L.bs, L.inv_t, out, nb, (long)nblk, st));
  } else if (which == DG_BLOCKS_NEIGHBOUR) {
    if (level < 1) return DG_ERR_INVALID;
    if (L.O16)
      CK(launch_unpack_bf16(L.O16, reinterpret_cast<float*>(out), nb, (long)nblk, st));
    else
      CK(launch_unpack_inverse<T>(L.O, L.cs, L.co_t, out, nb, (long)nblk, st));
  } else if (which == DG_BLOCKS_DIAG) {
    if (level == 0 && M.kind == DG_MESH_TRI)   // the fine-level probe again, at the stored state and shift
      CK(launch_probe_blocks_tri<T>(M, W, (T)sigma, out, (size_t)nb * nb, nullptr, 0, mg.lv[0].r, mg.lv[0].t, st));
    else if (level == 0)
      CK(launch_probe_blocks<T>(M, W, (T)sigma, out, (size_t)nb * nb, nullptr, 0, 0, mg.scratch, mg.scratch_elems,
                                st));
    else
      CK(launch_unpack_inverse<T>(L.Dop, L.cs, L.co_t, out, nb, (long)nblk, st));
  } else {
    return DG_ERR_INVALID;
  }
  CK(cudaStreamSynchronize(st));
  return DG_OK;
}

extern "C" dg_status dg_pmg_export_blocks(dg_pmg h, int level, int which, void* out, size_t out_bytes,
                                          void* stream) {
  if (!h || !out) return DG_ERR_INVALID;
  const Mesh& M = h->mesh->m;
  int nl = (int)(h->precision == DG_PREC_FP64 ? h->mg64.lv.size() : h->mg32.lv.size());
  if (level < 0 || level >= nl) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->precision == DG_PREC_FP64)
    return export_level<double>(h->mg64, M, h->mg64.W, h->sigma, level, which, (double*)out, out_bytes, st);
  return export_level<float>(h->mg32, M, h->mg32.W, h->sigma, level, which, (float*)out, out_bytes, st);
}

// ---------------------------------------------------------------- device-driven FGMRES cycle
namespace dgk {
// prm: [0] rtol, [1] atol, [2] ||b|| (set on cycle 0), [3] tol, [4] residual estimate, [5] cycle
// iq:  [0] iterations of this cycle, [1] stop reason (0 none yet, 1 converged, 2 non-finite,
//      3 iteration limit, 4 Krylov space exhausted)
__global__ void fgm_start_kernel(cudaGraphConditionalHandle h0, const double* res, int* kdim, double* prm, int* iq) {
  const double beta = res[1];
  if (prm[5] == 0.0) prm[2] = beta;
  const double tol = fmax(prm[0] * prm[2], prm[1]);
  prm[3] = tol;
  prm[4] = beta;
  iq[0] = 0;
  iq[1] = 0;
  const bool fin = isfinite(beta) != 0;
  const bool go = fin && beta > tol;
  if (!go) {
    kdim[0] = 0;
    iq[1] = fin ? 1 : 2;
  }
  cudaGraphSetConditional(h0, go ? 1u : 0u);
}

__global__ void fgm_check_kernel(cudaGraphConditionalHandle hn, int has_next, int j, int restart, const double* res,
                                 int* kdim, double* prm, int* iq) {
  const double r = res[0];
  prm[4] = r;
  iq[0] = j + 1;
  const bool nonfin = (kdim[1] & ST_NONFINITE) || !isfinite(r);
  const bool conv = !nonfin && r <= prm[3];
  const bool exhausted = kdim[0] <= j + 1 && j + 1 < restart;
  const bool stop = conv || nonfin || exhausted || j + 1 >= restart;
  if (stop) {
    if (kdim[0] > j + 1) kdim[0] = j + 1;
    iq[1] = conv ? 1 : (nonfin ? 2 : (exhausted ? 4 : 3));
  }
  if (has_next) cudaGraphSetConditional(hn, stop ? 0u : 1u);
}
}  // namespace dgk

// Last node of a graph (the node nothing depends on).
static cudaError_t last_node(cudaGraph_t g, cudaGraphNode_t* out) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  if (e != cudaSuccess || n == 0) return e != cudaSuccess ? e : cudaErrorInvalidValue;
  std::vector<cudaGraphNode_t> nodes(n);
  if ((e = cudaGraphGetNodes(g, nodes.data(), &n)) != cudaSuccess) return e;
  for (size_t i = 0; i < n; ++i) {
    size_t nd = 0;
    if ((e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd)) != cudaSuccess) return e;
    if (nd == 0) {
      *out = nodes[i];
      return cudaSuccess;
    }
  }
  return cudaErrorInvalidValue;
}

// One FGMRES iteration's work on the handle's capture stream (captured, not run):
// z_j = P^{-1} v_j (the preconditioner application), w = K z_j (exact FP64
// JVP at fgm_W), CGS2 + Givens.
static cudaError_t fgm_iteration(dg_pmg h, int j, cudaStream_t st) {
  const Mesh& M = h->mesh->m;
  const long N0 = (long)M.E * M.nb;
  Krylov<double>& K = h->outer;
  if (h->precision == DG_PREC_FP64) {
    CKE(h->mg64.apply(K.Vj(j), K.Zj(j), st));
  } else {
    CKE(launch_convert<double, float>(N0, K.Vj(j), h->r32, st));
    CKE(h->mg32.apply(h->r32, h->z32, st));
    CKE(launch_convert<float, double>(N0, h->z32, K.Zj(j), st));
  }
  CKE(launch_residual<double>(M, h->fgm_W, K.Zj(j), nullptr, h->fgm_sigma, true, K.w, st));
  return K.arnoldi(j, st);
}

// Build the cycle graph for `restart` iterations at shift sigma.
static cudaError_t build_fgm_graph(dg_pmg h, int restart, double sigma) {
  const long N0 = (long)h->mesh->m.E * h->mesh->m.nb;
  if (!h->fgm_W) {
    CKE(dalloc(h->allocs, (void**)&h->fgm_W, sizeof(double) * N0, &h->vector_bytes));
    CKE(dalloc(h->allocs, (void**)&h->fgm_r0, sizeof(double) * N0, &h->vector_bytes));
    CKE(dalloc(h->allocs, (void**)&h->fgm_dW, sizeof(double) * N0, &h->vector_bytes));
    CKE(dalloc(h->allocs, (void**)&h->fgm_prm, sizeof(double) * 8, &h->vector_bytes));
    CKE(dalloc(h->allocs, (void**)&h->fgm_iq, sizeof(int) * 4, &h->vector_bytes));
  }
  if (!h->cap_stream) CKE(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (h->fgm_exec) cudaGraphExecDestroy(h->fgm_exec);
  if (h->fgm_graph) cudaGraphDestroy(h->fgm_graph);
  h->fgm_exec = nullptr;
  h->fgm_graph = nullptr;
  h->fgm_sigma = sigma;
  h->fgm_restart = restart;
  cudaStream_t st = h->cap_stream;
  Krylov<double>& K = h->outer;
  cudaGraph_t g = nullptr;
  CKE(cudaGraphCreate(&g, 0));
  std::vector<cudaGraphConditionalHandle> hc(restart);
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < restart && e == cudaSuccess; ++j)
    e = cudaGraphConditionalHandleCreate(&hc[j], g, 0, cudaGraphCondAssignDefault);
  auto counter = [] { return __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED); };
  const unsigned long long l0 = counter();
  // head: v_0 = r0 / ||r0||, g = (||r0||, 0, ...), tolerance, open iteration 0
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t e1 = K.start(h->fgm_r0, st);
    if (e1 == cudaSuccess) {
      note_launch();
      fgm_start_kernel<<<1, 1, 0, st>>>(hc[0], K.res, K.kdim, h->fgm_prm, h->fgm_iq);
      e1 = cudaGetLastError();
    }
    cudaGraph_t gg = g;
    e = cudaStreamEndCapture(st, &gg);
    if (e == cudaSuccess) e = e1;
  }
  const unsigned long long l1 = counter();
  unsigned long long lb = 0;
  for (int j = 0; j < restart && e == cudaSuccess; ++j) {
    cudaGraphNode_t prev;
    if ((e = last_node(g, &prev)) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc[j];
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, &prev, nullptr, 1, &cp)) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const unsigned long long b0 = counter();
    if ((e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
      break;
    cudaError_t e1 = fgm_iteration(h, j, st);
    if (e1 == cudaSuccess) {
      note_launch();
      fgm_check_kernel<<<1, 1, 0, st>>>(j + 1 < restart ? hc[j + 1] : hc[j], j + 1 < restart ? 1 : 0, j, restart,
                                        K.res, K.kdim, h->fgm_prm, h->fgm_iq);
      e1 = cudaGetLastError();
    }
    cudaGraph_t bb = body;
    e = cudaStreamEndCapture(st, &bb);
    if (e == cudaSuccess) e = e1;
    lb = std::max(lb, counter() - b0);
  }
  const unsigned long long l2 = counter();
  // tail: dW += Z y over the effective Krylov dimension
  if (e == cudaSuccess) {
    cudaGraphNode_t prev;
    e = last_node(g, &prev);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(st, g, &prev, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t e1 = K.update(restart, h->fgm_dW, st);
      cudaGraph_t gg = g;
      e = cudaStreamEndCapture(st, &gg);
      if (e == cudaSuccess) e = e1;
    }
  }
  const unsigned long long l3 = counter();
  __atomic_fetch_sub(&launch_counter(), l3 - l0, __ATOMIC_RELAXED);   // captured, not run
  h->fgm_head_k = l1 - l0;
  h->fgm_body_k = lb;
  h->fgm_tail_k = l3 - l2;
  (void)l2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->fgm_exec, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->fgm_exec) cudaGraphExecDestroy(h->fgm_exec);
    cudaGraphDestroy(g);
    h->fgm_exec = nullptr;
    return e;
  }
  h->fgm_graph = g;
  return cudaSuccess;
}

// FGMRES with the exact JVP through the cycle graph: one host synchronisation
// per restart cycle.  Returns DG_ERR_UNSUPPORTED when the graph is not
// available (the caller then runs the host-driven loop).
static dg_status fgmres_graph(dg_pmg h, const double* W, const double* b, double sigma, const dg_krylov_opts* ko,
                              int restart, double* dW, dg_krylov_stats* stats, cudaStream_t st) {
  const char* env = getenv("DG_FGMRES_HOST");
  if (h->fgm_state < 0 || (env && env[0] == '1')) return DG_ERR_UNSUPPORTED;
  float ms_setup = 0.f;
  if (h->fgm_state == 0 || h->fgm_restart != restart || h->fgm_sigma != sigma) {
    const auto t0 = std::chrono::steady_clock::now();
    if (build_fgm_graph(h, restart, sigma) != cudaSuccess) {
      h->fgm_state = -1;
      return DG_ERR_UNSUPPORTED;
    }
    h->fgm_state = 1;
    ms_setup = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  const Mesh& M = h->mesh->m;
  const long N = (long)M.E * M.nb;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  CK(cudaMemcpyAsync(h->fgm_W, W, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->fgm_r0, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(h->fgm_dW, 0, sizeof(double) * N, st));
  double prm[8] = {ko->rtol, ko->atol, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  dg_status s = DG_OK;
  int iters = 0;
  double bnorm = 0.0, res = 0.0;
  bool converged = false;
  for (int cycle = 0; cycle <= ko->max_restarts; ++cycle) {
    prm[5] = (double)cycle;
    if (cycle > 0) {   // restart from the true residual b - K dW
      CK(launch_residual<double>(M, h->fgm_W, h->fgm_dW, nullptr, sigma, true, h->fgm_r0, st));
      CK(launch_axpby<double>(N, 1.0, b, -1.0, h->fgm_r0, st));
    }
    // the cycle's parameters (rtol, atol; ||b|| is kept from cycle 0)
    CK(cudaMemcpyAsync(h->fgm_prm, prm, sizeof(double) * 2, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->fgm_prm + 5, prm + 5, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaGraphLaunch(h->fgm_exec, st));
    double hp[8];
    int hq[4];
    CK(cudaMemcpyAsync(hp, h->fgm_prm, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hq, h->fgm_iq, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    __atomic_fetch_add(&launch_counter(), h->fgm_head_k + h->fgm_tail_k + (unsigned long long)hq[0] * h->fgm_body_k,
                       __ATOMIC_RELAXED);
    iters += hq[0];
    if (cycle == 0) bnorm = hp[2];
    res = hp[4];
    if (hq[1] == 2) {
      s = DG_ERR_BREAKDOWN;
      break;
    }
    if (hq[1] == 1 || hq[1] == 4) {
      converged = hq[1] == 1 || res <= hp[3];
      break;
    }
  }
  CK(cudaMemcpyAsync(dW, h->fgm_dW, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  cudaEventRecord(e1, st);
  float ms = 0.f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == DG_OK && !converged) s = DG_ERR_NOT_CONVERGED;
  if (s == DG_OK) {
    int hs = 0;
    cudaMemcpy(&hs, M.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (hs & ST_TIMEOUT) s = DG_ERR_TIMEOUT;
    else if (hs & ST_NONPHYSICAL) s = DG_ERR_NONPHYSICAL;
  }
  if (stats) {
    stats->iters = iters;
    stats->res0 = bnorm;
    stats->res_final = res;
    stats->rho = (iters > 0 && bnorm > 0) ? pow(res / bnorm, 1.0 / iters) : 0.0;
    stats->status = s;
    stats->ms_total = ms;
    stats->ms_setup = ms_setup;
  }
  return s;
}

extern "C" dg_status dg_fgmres_step(dg_mesh mesh, dg_pmg pmg, const double* W, const double* b, double sigma,
                                    const dg_krylov_opts* kopts, double* dW, dg_krylov_stats* stats,
                                    void* stream) {
  if (!mesh || !pmg || !W || !b || !kopts || !dW || dW == b || dW == W) return DG_ERR_INVALID;
  if (pmg->mesh != mesh) return DG_ERR_INVALID;
  const int restart = kopts->restart > 0 ? kopts->restart : 30;
  if (restart > pmg->outer_restart || kopts->max_restarts < 0 || !(kopts->rtol >= 0.0) || !(kopts->atol >= 0.0))
    return DG_ERR_INVALID;
  const int mode = kopts->jvp_mode;
  if (mode != DG_JVP_EXACT && mode != DG_JVP_FD && mode != DG_JVP_FD_SCALED) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == DG_JVP_EXACT && pmg->mesh->m.kind == DG_MESH_STRUCTURED) {
    // device-driven cycles: the convergence test runs on the device, the host
    // waits once per restart cycle
    dg_status gs = fgmres_graph(pmg, W, b, sigma, kopts, restart, dW, stats, st);
    if (gs != DG_ERR_UNSUPPORTED) return gs;
  }
  const Mesh& M = mesh->m;
  const long N = (long)M.E * M.nb;
  Krylov<double>& K = pmg->outer;
  double* RW = pmg->tmp64;            // R(W) for the FD mode
  double* rr = pmg->tmp64 + N;        // restart residual
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  auto kv = [&](const double* x, double* y) -> dg_status {
    if (mode == DG_JVP_EXACT) {
      CK(launch_residual<double>(M, W, x, nullptr, sigma, true, y, st));
    } else {
      CK(fd_jvp(M, W, RW, sigma, x, y, mode == DG_JVP_FD ? 0 : 1, st));
    }
    return DG_OK;
  };
  dg_status s = DG_OK;
  int iters = 0;
  double bnorm = 0, res = 0, host[3];
  bool converged = false;
  if (mode != DG_JVP_EXACT) {
    if (launch_residual<double>(M, W, nullptr, nullptr, 0.0, false, RW, st) != cudaSuccess) s = DG_ERR_CUDA;
  }
  if (s == DG_OK && cudaMemsetAsync(dW, 0, sizeof(double) * N, st) != cudaSuccess) s = DG_ERR_CUDA;
  for (int cycle = 0; s == DG_OK && cycle <= kopts->max_restarts && !converged; ++cycle) {
    const double* r0 = b;
    if (cycle > 0) {
      if ((s = kv(dW, rr)) != DG_OK) break;
      if (launch_axpby<double>(N, 1.0, b, -1.0, rr, st) != cudaSuccess) { s = DG_ERR_CUDA; break; }
      r0 = rr;
    }
    if (K.start(r0, st) != cudaSuccess) { s = DG_ERR_CUDA; break; }
    if (cudaMemcpyAsync(host, K.res + 1, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { s = DG_ERR_CUDA; break; }
    double beta = host[0];
    if (cycle == 0) bnorm = beta;
    const double tol = std::max(kopts->rtol * bnorm, kopts->atol);
    res = beta;
    if (!(beta > tol)) { converged = true; break; }
    int jdone = 0;
    for (int j = 0; j < restart; ++j) {
      if ((s = pmg_apply_impl(pmg, K.Vj(j), K.Zj(j), st)) != DG_OK) break;
      if ((s = kv(K.Zj(j), K.w)) != DG_OK) break;
      if (K.arnoldi(j, st) != cudaSuccess) { s = DG_ERR_CUDA; break; }
      ++iters;
      jdone = j + 1;
      int kd[2];
      if (cudaMemcpyAsync(host, K.res, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(kd, K.kdim, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) { s = DG_ERR_CUDA; break; }
      res = host[0];
      if (kd[1] & ST_NONFINITE || !isfinite(res)) { s = DG_ERR_BREAKDOWN; break; }
      if (res <= tol) { converged = true; break; }
      if (kd[0] <= j) { converged = res <= tol; break; }   // happy breakdown
    }
    if (s != DG_OK) break;
    if (K.update(jdone, dW, st) != cudaSuccess) { s = DG_ERR_CUDA; break; }
  }
  cudaEventRecord(e1, st);
  float ms = 0.f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == DG_OK && !converged) s = DG_ERR_NOT_CONVERGED;
  if (s == DG_OK) {
    int hs = 0;
    cudaMemcpy(&hs, M.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (hs & ST_TIMEOUT) s = DG_ERR_TIMEOUT;
    else if (hs & ST_NONPHYSICAL) s = DG_ERR_NONPHYSICAL;
  }
  if (stats) {
    stats->iters = iters;
    stats->res0 = bnorm;
    stats->res_final = res;
    stats->rho = (iters > 0 && bnorm > 0) ? pow(res / bnorm, 1.0 / iters) : 0.0;
    stats->status = s;
    stats->ms_total = ms;
    stats->ms_setup = 0.f;
  }
  return s;
}

namespace dgk {
unsigned long long& launch_counter() {
  static unsigned long long n = 0;
  return n;
}

// c = |J|/(2 dt); with geo (triangles: [E][5], |J| at 4) c is 1/(2 dt) and |J| per element
__global__ void bdf2_rhs_kernel(long N, const double* __restrict__ Wk, const double* __restrict__ Wn,
                                const double* __restrict__ Wnm1, double c, const double* __restrict__ geo, int nb,
                                double* __restrict__ b) {
  // on entry b holds R(Wk)
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
    const double ce = geo ? c * geo[(n / nb) * 5 + 4] : c;
    b[n] = -(ce * (3.0 * Wk[n] - 4.0 * Wn[n] + Wnm1[n]) + b[n]);
  }
}
}  // namespace dgk

extern "C" dg_status dg_bdf2_rhs(dg_mesh mesh, const double* Wk, const double* Wn, const double* Wnm1, double dt,
                                 double* b, void* stream) {
  if (!mesh || !Wk || !Wn || !Wnm1 || !b || b == Wk || b == Wn || b == Wnm1 || !(dt > 0.0)) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const Mesh& M = mesh->m;
  const long N = (long)M.E * M.nb;
  CK(launch_residual<double>(M, Wk, nullptr, nullptr, 0.0, false, b, st));
  int gr = (int)std::min<long>((N + 255) / 256, 4096);
  note_launch();
  const bool tri = M.kind == DG_MESH_TRI;
  bdf2_rhs_kernel<<<gr, 256, 0, st>>>(N, Wk, Wn, Wnm1, (tri ? 1.0 : M.detJ) / (2.0 * dt), tri ? M.tr64.geo : nullptr,
                                      M.nb, b);
  CK(cudaGetLastError());
  return DG_OK;
}

namespace dgk {
// b = -(c (Wk - Wn) + racc + b), b holding R(Wk) on entry; racc may be null
// c = sigma |J|, or sigma with |J| per element from geo (triangles)
__global__ void esdirk_rhs_kernel(long N, const double* __restrict__ Wk, const double* __restrict__ Wn,
                                  const double* __restrict__ racc, double c, const double* __restrict__ geo, int nb,
                                  double* __restrict__ b) {
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
    const double ce = geo ? c * geo[(n / nb) * 5 + 4] : c;
    b[n] = -(ce * (Wk[n] - Wn[n]) + (racc ? racc[n] : 0.0) + b[n]);
  }
}

// ESDIRK3 (four stages, third order, explicit first stage, stiffly accurate):
// Kennedy & Carpenter's ESDIRK3(2)4L[2]SA coefficients, as published.
constexpr double ES_G = 1767732205903.0 / 4055673282236.0;
constexpr double ES_A[4][4] = {
    {0.0, 0.0, 0.0, 0.0},
    {ES_G, ES_G, 0.0, 0.0},
    {2746238789719.0 / 10658868560708.0, -640167445237.0 / 6845629431997.0, ES_G, 0.0},
    {1471266399579.0 / 7840856788654.0, -4482444167858.0 / 7529755066697.0, 11266239266428.0 / 11593286722821.0,
     ES_G}};
}  // namespace dgk

extern "C" dg_status dg_esdirk3_rhs(dg_mesh mesh, const double* Wk, const double* Wn, double sigma,
                                    const double* racc, double* b, void* stream) {
  if (!mesh || !Wk || !Wn || !b || b == Wk || b == Wn || b == racc || !(sigma > 0.0)) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const Mesh& M = mesh->m;
  const long N = (long)M.E * M.nb;
  CK(launch_residual<double>(M, Wk, nullptr, nullptr, 0.0, false, b, st));
  int gr = (int)std::min<long>((N + 255) / 256, 4096);
  note_launch();
  const bool tri = M.kind == DG_MESH_TRI;
  esdirk_rhs_kernel<<<gr, 256, 0, st>>>(N, Wk, Wn, racc, sigma * (tri ? 1.0 : M.detJ), tri ? M.tr64.geo : nullptr,
                                        M.nb, b);
  CK(cudaGetLastError());
  return DG_OK;
}

extern "C" dg_status dg_esdirk3_step(dg_mesh mesh, dg_pmg pmg, const double* Wn, double dt, int newton,
                                     const dg_krylov_opts* kopts, double* work, size_t work_bytes, double* Wout,
                                     dg_krylov_stats* stats, void* stream) {
  if (!mesh || !pmg || !Wn || !kopts || !work || !Wout || Wout == Wn || !(dt > 0.0) || newton < 1 || newton > 16)
    return DG_ERR_INVALID;
  if (pmg->mesh != mesh) return DG_ERR_INVALID;
  const Mesh& M = mesh->m;
  const long N = (long)M.E * M.nb;
  if (work_bytes < sizeof(double) * 6 * (size_t)N) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  double* R[3] = {work, work + N, work + 2 * N};
  double* racc = work + 3 * N;
  double* b = work + 4 * N;
  double* dW = work + 5 * N;
  const double sigma = 1.0 / (ES_G * dt);
  dg_status s = dg_pmg_refresh(pmg, Wn, sigma, stream);   // lagged over the whole step
  if (s != DG_OK) return s;
  CK(launch_residual<double>(M, Wn, nullptr, nullptr, 0.0, false, R[0], st));
  CK(cudaMemcpyAsync(Wout, Wn, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  int iters = 0, solves = 0;
  dg_status worst = DG_OK;
  dg_krylov_stats last{};
  float ms = 0.f;
  for (int i = 1; i < 4; ++i) {
    for (int j = 0; j < i; ++j) CK(launch_axpby<double>(N, ES_A[i][j] / ES_A[i][i], R[j], j == 0 ? 0.0 : 1.0, racc, st));
    for (int it = 0; it < newton; ++it) {
      if ((s = dg_esdirk3_rhs(mesh, Wout, Wn, sigma, racc, b, stream)) != DG_OK) return s;
      s = dg_fgmres_step(mesh, pmg, Wout, b, sigma, kopts, dW, &last, stream);
      if (s != DG_OK && s != DG_ERR_NOT_CONVERGED) return s;
      if (s != DG_OK) worst = s;
      iters += last.iters;
      ms += last.ms_total;
      ++solves;
      CK(launch_axpby<double>(N, 1.0, dW, 1.0, Wout, st));
    }
    if (i < 3) CK(launch_residual<double>(M, Wout, nullptr, nullptr, 0.0, false, R[i], st));
  }
  CK(cudaStreamSynchronize(st));
  if (stats) {
    *stats = last;
    stats->iters = iters;
    stats->ms_total = ms;
    stats->status = worst;
  }
  (void)solves;
  return worst;
}

extern "C" dg_status dg_axpy(dg_mesh mesh, double alpha, const double* x, double* y, void* stream) {
  if (!mesh || !x || !y || x == y) return DG_ERR_INVALID;
  const long N = (long)mesh->m.E * mesh->m.nb;
  CK(launch_axpby<double>(N, alpha, x, 1.0, y, (cudaStream_t)stream));
  return DG_OK;
}

extern "C" dg_status dg_launch_count(unsigned long long* count) {
  if (!count) return DG_ERR_INVALID;
  *count = __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED);
  return DG_OK;
}
