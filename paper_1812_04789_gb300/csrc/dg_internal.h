// Internal declarations shared by the library's translation units: handle
// structures, kernel launchers and the Krylov workspace.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <vector>

#include "../../include/dg.h"
#include "dg_common.cuh"

namespace dgk {

enum : int { ST_NONPHYSICAL = 1, ST_SINGULAR = 2, ST_NONFINITE = 4, ST_TIMEOUT = 8 };

// Allow a kernel the device's largest dynamic shared memory (the per-block
// limit less its static shared memory).  Always the same value: host threads that launch one kernel for different meshes at once
// (serving workers) cannot overwrite each other's setting between setting it
// and launching.  The actual amount is still given per launch.
template <class K>
inline cudaError_t allow_max_smem(K kernel) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the per-block limit covers the kernel's static shared memory too
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smax - (int)fa.sharedSizeBytes);
}

// host-side count of kernel launches (dg_launch_count)
unsigned long long& launch_counter();
inline void note_launch() { __atomic_fetch_add(&launch_counter(), 1ULL, __ATOMIC_RELAXED); }

// Device tables of one precision (see MeshView for the layouts).
template <class T>
struct Tables {
  T *vphiT = nullptr, *vdphiT = nullptr, *vphi = nullptr, *vdphi = nullptr, *vw = nullptr;
  T *fphiT = nullptr, *fdphiT = nullptr, *fphi = nullptr, *fdphi = nullptr, *fw = nullptr;
  T* lift = nullptr;
  T* liftT = nullptr;        // lifted test tables [2d][2][nqf][nm]
  T* fpk = nullptr;          // packed face traces [2d][nm][nqf][4]
  T* fpw = nullptr;          // packed weighted face traces [2d][nqf][nm][4]
  T* slots = nullptr;        // face slots [E][d][2][nb]
  T* fd_w = nullptr;         // finite-difference JVP scratch: W + h v
  T* fd_r = nullptr;         // finite-difference JVP scratch: R(W + h v)
  T* fd_o = nullptr;         // FP32 JVP mode scratch: the product before conversion
  T* l1d = nullptr;          // Q space: L[p+1][nq1d], dL[p+1][nq1d] (reference), w[nq1d]
};

// Triangle-mesh tables of one precision (csrc/dg_tri.cu): per-triangle
// geometry and the reference basis on the collapsed rule and the edges.
template <class T>
struct TriTab {
  T *geo = nullptr, *egeo = nullptr;            // [E][5] inverse Jacobian + |J|; [E][3][3] normal, |J_F|
  T *vphi = nullptr, *vdphi = nullptr, *vw = nullptr;
  T *ephi = nullptr, *edphi = nullptr, *ew = nullptr, *P = nullptr;
};

enum : int { DG_MESH_STRUCTURED = 0, DG_MESH_TRI = 1 };

// Plan of the tensor-core block probe (FP32 blocks): seed variables are taken
// in groups of G whose accumulators, rows (w, v, i') x npad columns in
// 128-row tiles, fit the 512 TMEM columns; points are taken jq at a time,
// two points (8 K values: point x {value, d gradients, pad}) per MMA K step.
// Byte offsets of the shared-memory regions; ok = 0 when no plan fits.
struct TcPlan {
  int ok = 0;
  int G = 0, ngroups = 0, tiles = 0, npad = 0, nmp = 0, jq = 0, npv = 0, nks = 0, tmem_cols = 0;
  int oA = 0, oB = 0, oJ = 0, oT = 0, oW = 0, oU = 0, oFU = 0, smem = 0;
};
TcPlan tc_plan(int d, int nm, int nq, int nqf, int smem_max);

struct Mesh {
  dg_mesh_desc desc;
  dg_physics phys;
  int d, m, p, nq1d, nm, nb, nq, nqf, E;
  double h[3], detJ, faceJ[3];
  int* nbr = nullptr;        // device [E][d][2]
  Tables<double> t64;
  Tables<float> t32;
  TcPlan tc;                 // tensor-core probe plan and its element-independent tables:
  float* tc_test = nullptr;  //   test rows [point][kind][nmp] (weights, signs, lifting folded in)
  float* tc_trial = nullptr; //   trial operand per K step [nks][hi, lo][npad x 8] in MMA layout
  int* qidx = nullptr;       // Q space: mode index of the tensor index (a, b[, c]), a fastest-varying last
  int kind = DG_MESH_STRUCTURED;
  int* tnbr = nullptr;       // triangles: device [E][3] neighbour across each local edge
  int* tnbrf = nullptr;      //   and that neighbour's local edge
  TriTab<double> tr64;
  TriTab<float> tr32;
  int* tcolour = nullptr;    // triangles: device [E] greedy colouring (no two neighbours alike)
  int tncol = 0;
  int nfaces() const { return kind == DG_MESH_TRI ? 3 : 2 * d; }
  const int* face_nbr() const { return kind == DG_MESH_TRI ? tnbr : nbr; }   // [E][nfaces]
  int* status = nullptr;     // device status word
  double* scal = nullptr;    // device scalars for the FD JVP (norms, h)
  double* partials = nullptr;// reduction partials for the FD JVP norms
  std::vector<void*> allocs;
  template <class T> MeshView<T> view() const;
  template <class T> Phys<T> phys_t() const;
};

// ----------------------------------------------------------------- kernels
// Residual (jvp = false) or exact JVP (jvp = true) in precision T:
// out = [R(W) - S] or [sigma |J| V + dR/dW(W) V].
// For a JVP, Pv / Pf (optional, FP32 only) hold the primal traces of W from
// launch_primal_cache: the kernels then interpolate only V.  parts (structured
// meshes): 1 = the face kernel only, 2 = the volume kernel only (on the face
// slots as they are), 3 = both (the operation); parts other than 3 serve
// kernel timing.
template <class T>
cudaError_t launch_residual(const Mesh& M, const T* W, const T* V, const T* S, T sigma, bool jvp,
                            T* out, cudaStream_t st, const T* Pv = nullptr, const T* Pf = nullptr, int parts = 3);

// Blocks of a triangle mesh by coloured JVP probing (csrc/dg_tri.cu): D (row-
// major, dstride apart) = dR_e/dW_e + sigma |J_e| I; O (if given, row-major
// nbc^2 apart, [E][3]) the neighbour blocks on the modes of the first nmc.
template <class T>
cudaError_t launch_probe_blocks_tri(const Mesh& M, const T* W, T sigma, T* D, size_t dstride, T* O, int nmc,
                                    T* seed, T* out, cudaStream_t st);
// Residual / exact JVP on a triangle mesh (csrc/dg_tri.cu), same contract.
template <class T>
cudaError_t launch_residual_tri(const Mesh& M, const T* W, const T* V, const T* S, T sigma, bool jvp, T* out,
                                cudaStream_t st);
void free_mesh(Mesh& M);
// Look up the allocation-free residual's scratch array on the current device
// (csrc/dg_noalloc.cu); dg_mesh_create calls it so that the array exists
// before dg_residual_noalloc is first called.
dg_status noalloc_prepare();

// Volume part (+ face slots, + sigma |J| V or - S) by sum factorisation for the
// tensor-product space; cudaErrorNotSupported when the mesh is not Q_p or the
// element's stages do not fit shared memory (the direct kernel then runs).
template <class T>
cudaError_t launch_volume_q(const Mesh& M, const T* W, const T* V, const T* S, T sigma, bool jvp, T* out,
                            cudaStream_t st);

// Face term (the face slots) of the residual or exact JVP on a 3-D structured
// mesh by sum factorisation (csrc/dg_face_sf.cu); same contract as the face
// kernel of launch_residual (Pf: cached primal face traces, FP32 JVP only).
// cudaErrorNotSupported when the mesh is not 3-D or the stages do not fit.
template <class T>
cudaError_t launch_face_sf(const Mesh& M, const T* W, const T* V, T* slots, bool jvp, const T* Pf,
                           cudaStream_t st);

// Primal traces (u, grad u) of an FP32 state at the volume points and on both
// sides of every face point; primal_cache_sizes returns the volume cache's
// length and sets the face cache's (floats).
size_t primal_cache_sizes(const Mesh& M, size_t* nface);
cudaError_t launch_primal_cache(const Mesh& M, const float* W, float* Pv, float* Pf, cudaStream_t st);

// FP64 residual writing its face terms to `slots` (E * d * 2 * nb doubles)
// instead of the mesh handle's face-slot workspace.
cudaError_t launch_residual_with_slots(const Mesh& M, const double* W, const double* S, double* out,
                                       double* slots, cudaStream_t st);

// Element Jacobian blocks by probing: D[e] = dR_e/dW_e + sigma |J| I (nb x nb),
// and when O != nullptr the neighbour blocks O[e][2k+side] restricted to the
// first nmc modes of every variable (nbc x nbc, nbc = m nmc).
// D[e] starts at D + e * dstride (row-major, row stride nb).  With
// nbr_colmajor (FP32 only, probe_nbr_colmajor_ok) the neighbour blocks are
// written column-major by probe_nbr_kernel, else row-major, nbc^2 apart.
template <class T>
cudaError_t launch_probe_blocks(const Mesh& M, const T* W, T sigma, T* D, size_t dstride, T* O, int nmc,
                                int nbr_colmajor, T* scratch, size_t scratch_elems, cudaStream_t st);
template <class T>
size_t probe_scratch_elems(const Mesh& M, int nmc, bool* fits_smem);

// Tensor-core probe of the FP32 diagonal blocks: D[e] = dR_e/dW_e (volume and
// own-face seeds) + sigma |J| I, written in full.  Neighbour-seeded terms are
// the SIMT kernel's.  build_tc_tables fills the mesh's tables (M.tc.ok).
cudaError_t launch_probe_tc(const Mesh& M, const float* W, float sigma, float* D, size_t dstride,
                            cudaStream_t st);
cudaError_t build_tc_tables(Mesh& M);

// FP32 neighbour blocks O[e][2k+side] (first nmc modes per variable, row-major
// nbc x nbc) for meshes with the tensor-core probe tables and no direction of
// one element; probe_nbr_fits says whether the kernel applies.
// colmajor: blocks column-major with leading dimension inv_ld(nbc), nbc *
// inv_ld(nbc) apart (else row-major, nbc^2 apart).
bool probe_nbr_fits(const Mesh& M, int nmc);
cudaError_t launch_probe_nbr(const Mesh& M, const float* W, float* O, int nmc, int colmajor, cudaStream_t st);
// Whether the FP32 neighbour blocks of this mesh come from probe_nbr_kernel
// (tensor-core tables present, the kernel applies, not disabled by DG_PROBE_SIMT).
bool probe_nbr_colmajor_ok(const Mesh& M, int nmc);

// Batched in-place inverse of nblk row-major blocks of size nb starting bstride
// elements apart (bstride >= nb * inv_ld(nb)).  *transposed = 1 when the
// inverse is stored column-major with leading dimension inv_ld(nb) (rows
// padded to a 16-byte multiple, the layout the block-Jacobi apply streams with
// vector loads), 0 when it stays row-major (blocks too large for registers or
// shared memory).  Gauss-Jordan, partial pivoting.
template <class T>
constexpr int inv_ld(int nb) {
  return (nb + (int)(16 / sizeof(T)) - 1) / (int)(16 / sizeof(T)) * (int)(16 / sizeof(T));
}
template <class T>
cudaError_t launch_block_inverse(T* A, int nb, size_t bstride, long nblk, int* status, int* transposed,
                                 cudaStream_t st);

// Leading sub-block per variable pair: dst[b] (m nmt)^2 from src[b] (m nms)^2.
// Blocks start sstride / dstride elements apart; *_t = 1: column-major with
// leading dimension inv_ld(nb), 0: row-major (row stride nb).
template <class T>
cudaError_t launch_truncate_blocks(const T* src, int nms, size_t sstride, int src_t, T* dst, int nmt,
                                   size_t dstride, int dst_t, int m, long nblk, cudaStream_t st);

// z[e] = Ainv[e] r[e]; blocks bstride apart, column-major with leading
// dimension inv_ld(nb) when transposed, else row-major.
template <class T>
cudaError_t launch_block_apply(const T* A, size_t bstride, int transposed, const T* r, T* z, int nb, int E,
                               cudaStream_t st);

// Row-major copy (nb x nb per block, packed) of inverse blocks in the layout above.
template <class T>
cudaError_t launch_unpack_inverse(const T* A, size_t bstride, int transposed, T* out, int nb, long nblk,
                                  cudaStream_t st);

// BF16 block storage (mixed precision): column-major, leading dimension
// ld_bf16(nb) = nb rounded up to 8 (16 bytes), nb * ld_bf16(nb) entries per
// block, padding rows zero.  launch_to_bf16 rounds FP32 blocks (layout as in
// launch_block_apply: column-major with inv_ld<float>(nb) when src_t, else
// row-major) to nearest; the apply and BSR kernels multiply in FP32.
constexpr int ld_bf16(int nb) { return (nb + 7) / 8 * 8; }
cudaError_t launch_to_bf16(const float* src, size_t sstride, int src_t, unsigned short* dst, int nb, long nblk,
                           cudaStream_t st);
cudaError_t launch_unpack_bf16(const unsigned short* A, float* out, int nb, long nblk, cudaStream_t st);
cudaError_t launch_block_apply_bf16(const unsigned short* A, const float* r, float* z, int nb, int E,
                                    cudaStream_t st);
cudaError_t launch_bsr_bf16(const unsigned short* D, const unsigned short* O, const int* nbr, int nf,
                            const float* x, float* y, int nb, int E, cudaStream_t st);

// y = D x + sum_s O_s x_nbr(s); blocks bstride apart (D: [E], O: [E][2d]),
// column-major with leading dimension inv_ld(nb) when transposed.
template <class T>
cudaError_t launch_bsr(const T* D, const T* O, size_t bstride, int transposed, const int* nbr, int d,
                       const T* x, T* y, int nb, int E, cudaStream_t st);

// vector helpers
template <class T> cudaError_t launch_axpby(long n, double a, const T* x, double b, T* y, cudaStream_t st);
template <class A, class B> cudaError_t launch_convert(long n, const A* x, B* y, cudaStream_t st);
template <class T> cudaError_t launch_restrict(const T* xf, int nmf, T* xc, int nmc, long nev, cudaStream_t st);
template <class T> cudaError_t launch_prolong(const T* xc, int nmc, T* xf, int nmf, long nev, bool add, cudaStream_t st);

// ----------------------------------------------------------------- Krylov
// Right-preconditioned (F)GMRES workspace on the device.  All scalars (H, g,
// Givens, y, residual) stay in device memory; nothing is read back unless
// the host asks for the residual estimate.
template <class T>
struct Krylov {
  long N = 0;
  int nmax = 0;
  int G = 0;                 // reduction CTAs (fixed => deterministic sums)
  T* V = nullptr;            // (nmax+1) x N
  T* Z = nullptr;            // nmax x N
  T* w = nullptr;            // N
  double* H = nullptr;       // (nmax+1) x nmax, column-major
  double* cs = nullptr;
  double* sn = nullptr;
  double* g = nullptr;       // nmax+1
  double* y = nullptr;       // nmax
  double* part = nullptr;    // (nmax+1) x G reduction partials
  double* res = nullptr;     // residual estimate |g[j+1]|
  int* kdim = nullptr;       // [0] effective Krylov dimension (breakdown), [1] status bits
  std::vector<void*> allocs;
  cudaError_t alloc(long N, int nmax);
  void release();
  size_t bytes() const;
  // v0 = r / ||r||, g = (||r||, 0, ...)
  cudaError_t start(const T* r, cudaStream_t st);
  // after w = A z_j (w holds it): CGS2 against V[0..j], normalise into V[j+1],
  // Givens update of column j; writes |g[j+1]| to res
  cudaError_t arnoldi(int j, cudaStream_t st);
  // x += Z y with H[:k,:k] y = g[:k], k = min(kdone, kdim)
  cudaError_t update(int kdone, T* x, cudaStream_t st);
  T* Vj(int j) { return V + (size_t)j * N; }
  T* Zj(int j) { return Z + (size_t)j * N; }
};

// ----------------------------------------------------------------- pMG
// Launch plan of the persistent coarse-level smoother (csrc/dg_smoother.cu):
// grid CTAs (all co-resident, cooperative launch), chunk elements per CTA,
// epc elements per pass of the block-sparse product, tpe threads per block,
// dynamic shared memory for up to nu_max iterations.  ok = 0: not available.
struct CoopPlan {
  int ok = 0, grid = 0, chunk = 0, epc = 0, tpe = 0, nu_max = 0;
  size_t smem = 0;
};
cudaError_t plan_coop_smoother(int bf16, int nb, int nf, int E, int nu, CoopPlan* plan);
constexpr int COOP_BAR_WORDS = 64;   // barrier words per level (arrivals at 0, release at 32)
// One SMOOTH call (nu GMRES(BJ) iterations from x on A x = b, Algorithm 2) in
// one cooperative launch: FP32 vectors, blocks column-major in FP32 (inv_ld)
// or, when Dinv16 is given, BF16 (ld_bf16).  part: grid * (2 (nu_max + 1) + 1)
// doubles; bar: COOP_BAR_WORDS words (zeroed by the call, on the stream); a bounded
// grid barrier that runs out sets ST_TIMEOUT in *status.  expect_extra > 0
// makes every barrier wait for CTAs that do not exist (the wait then runs out).
cudaError_t launch_coop_smoother(const CoopPlan& pl, const float* Dinv, const float* Dop, const float* O,
                                 const unsigned short* Dinv16, const unsigned short* Dop16, const unsigned short* O16,
                                 const int* nbr, int nf, const float* b, float* x, int nu, Krylov<float>& K,
                                 double* part, unsigned* bar, int* status, int expect_extra, int nb, int E,
                                 cudaStream_t st);

template <class T>
struct Level {
  int p = 0, nm = 0, nb = 0;
  long N = 0;
  T* Dinv = nullptr;         // inverse diagonal blocks, E blocks bs apart (see launch_block_inverse)
  size_t bs = 0;             // block stride of Dinv: nb * inv_ld<T>(nb)
  int inv_t = 0;             // Dinv column-major (1) or row-major (0)
  T* Dop = nullptr;          // diagonal blocks of the inherited operator (l >= 1)
  T* O = nullptr;            // neighbour blocks [E][2d] (l >= 1)
  int co_t = 0;              // Dop and O column-major (1, leading dimension inv_ld(nb)) or row-major
  size_t cs = 0;             // block stride of Dop and O
  T *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
  int nu_pre = 0, nu_post = 0;
  Krylov<T> kr;
  // BF16 copies the smoother streams instead (mixed precision, DG_STORE_BF16):
  // inverse diagonal blocks, inherited diagonal and neighbour blocks (l >= 1)
  unsigned short* Dinv16 = nullptr;
  unsigned short* Dop16 = nullptr;
  unsigned short* O16 = nullptr;
  CoopPlan coop;             // persistent smoother (FP32 coarse levels), when available
  double* cpart = nullptr;   //   its reduction partials [grid][2 (nu + 1) + 1], then the totals
  unsigned* cbar = nullptr;  //   and barrier counter
};

template <class T>
struct MG {
  const Mesh* mesh = nullptr;
  std::vector<Level<T>> lv;
  T* W = nullptr;            // state in precision T (fine JVP operator)
  T sigma = 0;
  int nu_coarse = 0;
  int cycle = 0;
  T* scratch = nullptr;      // probing caches in global memory (large blocks only)
  size_t scratch_elems = 0;
  T* Pv = nullptr;           // primal traces of W for the fine JVPs (mixed precision;
  T* Pf = nullptr;           //   refreshed with the blocks), else null
  std::vector<void*> allocs;
  // element block ILU(0) preconditioning the coarsest smoother (DG_COARSE_BILU)
  int bilu = 0, bl_kind = 0;  // on / DG_ORDER_* of the element order
  T* Sinv = nullptr;          // [E][nb][nb] row-major: inverses of the ILU(0) pivot blocks
  int* bl_pos = nullptr;      // device [E]: position of every element in the order
  int* bl_ptr = nullptr;      // device [E + 1]: level l = bl_el[bl_ptr[l] .. bl_ptr[l + 1])
  int* bl_el = nullptr;       // device [E]: elements by level, in order within a level
  int* bl_nlev = nullptr;     // device [1]: number of levels (read by the kernels)
  double* bl_c = nullptr;     // device [E][2d]: MDF reduced weights
  int bl_warps = 0, bl_chunk = 0, bl_resident = 0;   // launch plan (bilu_plan)
  std::vector<int> h_nbr, h_order, h_level, h_ptr, h_el, h_pos;
  std::vector<double> h_c;
  int h_nlev = 0, h_nlev_buf = 0;
  int coop_extra = 0;         // test hook: extra barrier arrivals the persistent smoother waits for
  cudaError_t op(int l, const T* x, T* y, cudaStream_t st);
  cudaError_t smooth(int l, const T* b, T* x, int nu, cudaStream_t st);
  cudaError_t mg_v(int l, cudaStream_t st);           // on lv[l].b, lv[l].x
  cudaError_t apply(const T* r, T* z, cudaStream_t st);
};

// Element block ILU(0) of the coarsest level (csrc/dg_bilu.cu).  bilu_order_host:
// the host ordering of dg_bilu_order, returns the level count or -1.
// bilu_plan: launch plan for the level's block size (false: too large).
// bilu_refresh: order (MDF: from the level's blocks, one device-to-host copy
// and a host synchronisation; natural / colour: once) and factorisation, after
// the level's blocks and inverses.  launch_bilu_apply: z = (L U)^{-1} r.
int bilu_order_host(int E, int nf, const int* nbr, const double* c, int kind, int* order, int* level);
template <class T>
bool bilu_plan(MG<T>& mg);
template <class T>
cudaError_t bilu_refresh(MG<T>& mg, cudaStream_t st);
template <class T>
cudaError_t launch_bilu_apply(const MG<T>& mg, const T* r, T* z, cudaStream_t st);

}  // namespace dgk

struct dg_mesh_s {
  dgk::Mesh m;
};

struct dg_pmg_s {
  dg_mesh mesh = nullptr;
  dg_pmg_opts opts;
  double sigma = 0;
  int precision = 0;
  dgk::MG<double> mg64;
  dgk::MG<float> mg32;
  double* r_in = nullptr;    // staging for mixed precision
  float* r32 = nullptr;
  float* z32 = nullptr;
  dgk::Krylov<double> outer; // FGMRES workspace (allocated at first solve)
  int outer_restart = 0;
  double* tmp64 = nullptr;
  double* r64 = nullptr;     // FP64 staging of the preconditioner input/output
  double* z64 = nullptr;
  // the whole preconditioner application, captured once as a CUDA graph on
  // fixed staging buffers and replayed on the caller's stream
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  unsigned long long graph_kernels = 0;
  double graph_sigma = 0;    // the shift the graph was captured with (a by-value kernel argument)
  // one FGMRES cycle (exact JVP) as a graph: the head, `restart` iterations
  // each behind a conditional (IF) node that the previous iteration's
  // convergence check opens or leaves shut, and the solution update; it works
  // on staging vectors so the caller's pointers can change between solves
  cudaGraph_t fgm_graph = nullptr;
  cudaGraphExec_t fgm_exec = nullptr;
  int fgm_state = 0;          // 0: not built, 1: ready, -1: not available (host-driven loop)
  int fgm_restart = 0;
  double fgm_sigma = 0;
  double* fgm_W = nullptr;    // the linearisation state
  double* fgm_r0 = nullptr;   // the cycle's starting residual (b, or b - K dW after a restart)
  double* fgm_dW = nullptr;   // the solution, accumulated over cycles
  double* fgm_prm = nullptr;  // device scalars: rtol, atol, ||b||, tol, residual estimate, cycle
  int* fgm_iq = nullptr;      // device ints: iterations of the cycle, stop reason
  unsigned long long fgm_head_k = 0, fgm_body_k = 0, fgm_tail_k = 0;   // kernels per part (launch accounting)
  std::vector<void*> allocs;
  size_t block_bytes = 0, vector_bytes = 0;
};
