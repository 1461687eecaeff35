// Serving runtime: continuous admission of implicit-step requests.
//
// A request is one BDF2 implicit step (the form of eq. NEWTON / eq. ODEDG with
// the BDF2 shift) of one case: mesh, physics, order, p-multigrid levels and
// precision, state W^n and W^{n-1} in host memory, dt, Newton iterations.
// Requests are admitted into slots as memory frees up: a slot owns a mesh
// handle, a p-multigrid handle (preconditioner + Krylov workspace) and device
// vectors, and stays resident after its request completes, so a later request
// of the same shape reuses it (only the preconditioner is refreshed).  The sum
// of the resident slots' device bytes never exceeds the budget; idle slots are
// evicted least-recently-used to make room.  Each worker thread runs one
// request at a time on its slot's own stream, so the device interleaves the
// work of all in-flight requests.  Results are bitwise independent of the mix:
// every kernel is deterministic and a slot's computation touches only its own
// buffers.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <vector>
#include <algorithm>

#include "dg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Key {
  dg_mesh_desc desc;
  dg_physics phys;
  dg_pmg_opts opts;
  bool operator==(const Key& o) const {
    // field by field: the descriptor has tail padding a caller need not clear
    const dg_mesh_desc& a = desc;
    const dg_mesh_desc& b = o.desc;
    bool same = a.dim == b.dim && a.p == b.p && a.nq1d == b.nq1d && a.space == b.space;
    for (int k = 0; k < 3; ++k) same = same && a.n[k] == b.n[k] && a.lo[k] == b.lo[k] && a.hi[k] == b.hi[k];
    return same && memcmp(&phys, &o.phys, sizeof(phys)) == 0 && memcmp(&opts, &o.opts, sizeof(opts)) == 0;
  }
};

struct Slot {
  Key key;
  dg_mesh mesh = nullptr;
  dg_pmg pmg = nullptr;
  cudaStream_t stream = nullptr;
  double *Wn = nullptr, *Wnm1 = nullptr, *Wk = nullptr, *b = nullptr, *dW = nullptr;
  size_t ndofs = 0;
  size_t bytes = 0;
  bool busy = false;
  unsigned long long last_use = 0;
};

struct Job {
  long long id;
  Key key;
  const double* Wn;
  const double* Wnm1;
  double* Wout;
  double dt;
  int newton;
  double rtol;
  Clock::time_point t_submit;
};

struct Done {
  long long id;
  int status;
  double latency_ms;
  double queue_ms;
  int fgmres_iters;
  long long ndofs;
};

// Conservative device-memory estimate of a slot (bytes), from the sizes the
// mesh and p-multigrid handles allocate.
size_t estimate_bytes(const Key& k) {
  const dg_mesh_desc& d = k.desc;
  long E = 1;
  for (int i = 0; i < d.dim; ++i) E *= d.n[i];
  auto nmodes = [&](int p) {
    long c = 1;
    for (int i = 1; i <= d.dim; ++i) c = d.space == DG_SPACE_Q ? c * (p + 1) : c * (p + i) / i;
    return c;
  };
  const int m = d.dim + 2;
  const long nm0 = nmodes(d.p), nb0 = m * nm0, N0 = E * nb0;
  const size_t es = k.opts.precision == DG_PREC_MIXED ? 4 : 8;
  size_t bytes = 0;
  bytes += (size_t)E * d.dim * 2 * nb0 * (8 + 4);          // face slots (FP64 + FP32)
  bytes += (size_t)N0 * (8 + 4) * 2;                        // FD scratch
  bytes += (size_t)N0 * 8 * 5;                              // the slot's own vectors
  const int restart = k.opts.fgmres_restart > 0 ? k.opts.fgmres_restart : 30;
  bytes += (size_t)N0 * 8 * (2 * restart + 6);              // outer FGMRES + staging
  const int nl = k.opts.cycle == DG_CYCLE_BJ ? 1 : k.opts.n_levels;
  for (int l = 0; l < nl; ++l) {
    long nb = m * nmodes(k.opts.p_level[l]);
    const long ld = (nb + (long)(16 / es) - 1) / (long)(16 / es) * (long)(16 / es);   // padded inverse rows
    bytes += (size_t)E * nb * ld * es * (l == 0 ? 1 : 2 + 2 * d.dim);   // inverse (+ coarse D and O)
    if (k.opts.block_storage == DG_STORE_BF16)                          // their BF16 copies
      bytes += (size_t)E * nb * ((nb + 7) / 8 * 8) * 2 * (l == 0 ? 1 : 2 + 2 * d.dim);
    int nu = l == nl - 1 ? k.opts.nu_coarse : std::max(k.opts.nu_pre[l], k.opts.nu_post[l]);
    bytes += (size_t)E * nb * es * (2 * nu + 8);
  }
  if (k.opts.coarse_precond == DG_COARSE_BILU && nl >= 2) {   // block ILU(0) pivot inverses + order
    const long nbc = m * nmodes(k.opts.p_level[nl - 1]);
    bytes += (size_t)E * nbc * nbc * es + (size_t)E * (2 * d.dim * 8 + 16);
  }
  if (k.opts.precision == DG_PREC_MIXED && k.opts.cycle != DG_CYCLE_BJ) {   // primal-trace caches
    const int nq1 = d.nq1d > 0 ? d.nq1d : d.p + 2;
    long nq = 1, nqf = 1;
    for (int i = 0; i < d.dim; ++i) nq *= nq1;
    for (int i = 1; i < d.dim; ++i) nqf *= nq1;
    bytes += (size_t)E * (nq + 2 * d.dim * nqf) * m * (1 + d.dim) * 4;
  }
  return bytes + (64u << 20);                               // tables, probing scratch, slack
}

}  // namespace

struct dg_server_s {
  size_t budget = 0;
  size_t used = 0;
  int device = 0;
  std::vector<Slot*> slots;
  std::deque<Job> queue;
  std::vector<Done> done;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  unsigned long long tick = 0;
  long long submitted = 0, completed = 0;
};

namespace {

void free_slot(Slot* s) {
  if (s->pmg) dg_pmg_destroy(s->pmg);
  if (s->mesh) dg_mesh_destroy(s->mesh);
  for (double* p : {s->Wn, s->Wnm1, s->Wk, s->b, s->dW})
    if (p) cudaFree(p);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

// Build the slot's handles and buffers at the job's state and shift (called by
// its worker, outside the lock).
dg_status build_slot(Slot* s, const double* Wn_host, double sigma) {
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return DG_ERR_CUDA;
  dg_status st = dg_mesh_create(&s->key.desc, &s->key.phys, s->stream, &s->mesh);
  if (st != DG_OK) return st;
  int E = 0, nm = 0, m = 0;
  dg_mesh_info(s->mesh, &E, &nm, &m, &s->ndofs);
  for (double** p : {&s->Wn, &s->Wnm1, &s->Wk, &s->b, &s->dW})
    if (cudaMalloc((void**)p, s->ndofs * sizeof(double)) != cudaSuccess) return DG_ERR_OOM;
  if (cudaMemcpyAsync(s->Wn, Wn_host, s->ndofs * sizeof(double), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    return DG_ERR_CUDA;
  return dg_pmg_setup(s->mesh, s->Wn, sigma, &s->key.opts, s->stream, &s->pmg);
}

// One BDF2 implicit step on the slot (Newton with the preconditioner lagged at
// W^n; a freshly built slot already holds it).
dg_status run_step(Slot* s, const Job& j, bool fresh, int* iters) {
  cudaStream_t st = s->stream;
  const size_t bytes = s->ndofs * sizeof(double);
  if (cudaMemcpyAsync(s->Wn, j.Wn, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return DG_ERR_CUDA;
  if (cudaMemcpyAsync(s->Wnm1, j.Wnm1, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return DG_ERR_CUDA;
  const double sigma = 1.5 / j.dt;
  dg_status r = fresh ? DG_OK : dg_pmg_refresh(s->pmg, s->Wn, sigma, st);
  if (r != DG_OK) return r;
  if (cudaMemcpyAsync(s->Wk, s->Wn, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return DG_ERR_CUDA;
  dg_krylov_opts ko;
  ko.restart = s->key.opts.fgmres_restart > 0 ? s->key.opts.fgmres_restart : 30;
  ko.max_restarts = 4;
  ko.rtol = j.rtol;
  ko.atol = 0.0;
  ko.jvp_mode = DG_JVP_EXACT;
  *iters = 0;
  for (int it = 0; it < j.newton; ++it) {
    if ((r = dg_bdf2_rhs(s->mesh, s->Wk, s->Wn, s->Wnm1, j.dt, s->b, st)) != DG_OK) return r;
    dg_krylov_stats ks;
    r = dg_fgmres_step(s->mesh, s->pmg, s->Wk, s->b, sigma, &ko, s->dW, &ks, st);
    *iters += ks.iters;
    if (r != DG_OK) return r;
    if ((r = dg_axpy(s->mesh, 1.0, s->dW, s->Wk, st)) != DG_OK) return r;
  }
  if (cudaMemcpyAsync(j.Wout, s->Wk, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return DG_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DG_ERR_CUDA;
  return dg_status_sync(s->mesh, st);
}

void worker_main(dg_server_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Job job;
    Slot* slot = nullptr;
    bool fresh = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) return;
        // take the first queued job that can be placed now (continuous admission)
        bool placed = false, rescan = false;
        for (auto it = S->queue.begin(); it != S->queue.end() && !placed; ++it) {
          Slot* hit = nullptr;
          for (Slot* s : S->slots)
            if (!s->busy && s->key == it->key) hit = s;
          if (hit) {
            slot = hit;
            placed = true;
          } else {
            size_t need = estimate_bytes(it->key);
            // evict idle slots of other shapes, least recently used first
            while (S->used + need > S->budget) {
              Slot* lru = nullptr;
              for (Slot* s : S->slots)
                if (!s->busy && (!lru || s->last_use < lru->last_use)) lru = s;
              if (!lru) break;
              S->slots.erase(std::find(S->slots.begin(), S->slots.end(), lru));
              S->used -= lru->bytes;
              free_slot(lru);
            }
            if (S->used + need <= S->budget) {
              slot = new Slot();
              slot->key = it->key;
              slot->bytes = need;
              S->used += need;
              S->slots.push_back(slot);
              fresh = true;
              placed = true;
            } else if (S->slots.empty() && need > S->budget) {
              // can never fit: fail it
              S->done.push_back(Done{it->id, DG_ERR_OOM, 0.0, 0.0, 0, 0});
              ++S->completed;
              S->queue.erase(it);
              S->cv_done.notify_all();
              rescan = true;
              break;
            }
          }
          if (placed) {
            job = *it;
            S->queue.erase(it);
            break;
          }
        }
        if (placed) {
          slot->busy = true;
          slot->last_use = ++S->tick;
          break;
        }
        if (rescan) continue;
        S->cv_work.wait(lk);
      }
    }
    Clock::time_point t_start = Clock::now();
    dg_status st = DG_OK;
    if (fresh) st = build_slot(slot, job.Wn, 1.5 / job.dt);
    int iters = 0;
    if (st == DG_OK) st = run_step(slot, job, fresh, &iters);
    Clock::time_point t_end = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      Done d;
      d.id = job.id;
      d.status = st;
      d.latency_ms = std::chrono::duration<double, std::milli>(t_end - job.t_submit).count();
      d.queue_ms = std::chrono::duration<double, std::milli>(t_start - job.t_submit).count();
      d.fgmres_iters = iters;
      d.ndofs = (long long)slot->ndofs;
      S->done.push_back(d);
      ++S->completed;
      slot->busy = false;
      if (st != DG_OK) {
        // a failed slot is not reused
        S->slots.erase(std::find(S->slots.begin(), S->slots.end(), slot));
        S->used -= slot->bytes;
        free_slot(slot);
      }
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" dg_status dg_server_create(size_t budget_bytes, int workers, dg_server* out) {
  if (!out) return DG_ERR_INVALID;
  *out = nullptr;
  if (workers < 1 || workers > 64 || budget_bytes == 0) return DG_ERR_INVALID;
  dg_server S = new dg_server_s();
  S->budget = budget_bytes;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return DG_ERR_CUDA;
  }
  for (int i = 0; i < workers; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return DG_OK;
}

extern "C" dg_status dg_server_submit(dg_server S, long long id, const dg_mesh_desc* desc, const dg_physics* phys,
                                      const dg_pmg_opts* opts, const double* Wn, const double* Wnm1, double dt,
                                      int newton, double rtol, double* Wout) {
  if (!S || !desc || !phys || !opts || !Wn || !Wnm1 || !Wout || !(dt > 0.0) || newton < 1 || !(rtol > 0.0))
    return DG_ERR_INVALID;
  Job j;
  j.id = id;
  memset(&j.key, 0, sizeof(j.key));
  j.key.desc = *desc;
  j.key.phys = *phys;
  j.key.opts = *opts;
  j.Wn = Wn;
  j.Wnm1 = Wnm1;
  j.Wout = Wout;
  j.dt = dt;
  j.newton = newton;
  j.rtol = rtol;
  j.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->queue.push_back(j);
    ++S->submitted;
  }
  S->cv_work.notify_all();
  return DG_OK;
}

// Wait until at least `min_done` completions are available (or timeout_ms
// passes), then copy up to `cap` completion records out (oldest first).
extern "C" dg_status dg_server_poll(dg_server S, int min_done, int timeout_ms, dg_server_result* out, int cap,
                                    int* n_out) {
  if (!S || !n_out || (cap > 0 && !out)) return DG_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&] { return (int)S->done.size() >= min_done; };
  bool ok;
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, ready);
    ok = true;
  } else {
    ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  int n = std::min(cap, (int)S->done.size());
  for (int i = 0; i < n; ++i) {
    out[i].id = S->done[i].id;
    out[i].status = S->done[i].status;
    out[i].latency_ms = S->done[i].latency_ms;
    out[i].queue_ms = S->done[i].queue_ms;
    out[i].fgmres_iters = S->done[i].fgmres_iters;
    out[i].ndofs = S->done[i].ndofs;
  }
  S->done.erase(S->done.begin(), S->done.begin() + n);
  *n_out = n;
  return ok ? DG_OK : DG_ERR_TIMEOUT;
}

extern "C" dg_status dg_server_stats(dg_server S, size_t* used_bytes, int* resident_slots, long long* submitted,
                                     long long* completed) {
  if (!S) return DG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  if (used_bytes) *used_bytes = S->used;
  if (resident_slots) *resident_slots = (int)S->slots.size();
  if (submitted) *submitted = S->submitted;
  if (completed) *completed = S->completed;
  return DG_OK;
}

extern "C" dg_status dg_server_destroy(dg_server S) {
  if (!S) return DG_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (Slot* s : S->slots) free_slot(s);
  delete S;
  return DG_OK;
}
