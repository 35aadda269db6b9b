// Serving: continuous batching of independent polarization solves on one GPU
// (C ABI amp_server_*, declared in include/amoebapol.h). The paper has no
// serving counterpart; its throughput runs are many MPI ranks on one system
// (Section "Parallel performance").
//
// Host side, all native:
//   - a batch driver thread owns the batched engine of amp_batch.cu (small
//     clusters): it admits requests into the arena between iterations,
//     launches one pair of persistent kernels per iteration for every request
//     in flight, reads the requests' end records one iteration behind (so the
//     GPU always has the next iteration queued), and copies finished dipoles
//     out;
//   - n_workers worker threads, each with its own CUDA stream, run the other
//     requests through the single-system calls (amp_set_system ...
//     amp_polarization_energy) on contexts from a pool keyed by PME grid
//     size;
//   - admission by memory: the contexts' actual bytes, an upper estimate for
//     a context that must be created, the arena, the resident dipoles.
// Requests are independent: each one's arithmetic is that of a solve alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "amp_batch.cuh"
#include "amp_internal.cuh"

namespace amp {
namespace serve {

using Clock = std::chrono::steady_clock;

struct Request {
  long long ticket = 0;
  int n = 0;
  double box = 0.0, cutoff = 0.0, beta = 0.0;
  int grid = 0;
  std::vector<double> xyz, q, dip, quad, alpha, thole;
  std::vector<int> mol;
  std::string key;
  long long est_bytes = 0;
  // result
  bool done = false;
  std::vector<double> mu;
  amp_server_result res{};
};

// Cutoff, beta and grid of a periodic request box: the caller's when given,
// else cutoff = min(7, L/2 - 1e-6), beta = 3.8122/cutoff (erfc(beta cutoff)
// = 7e-8, as 0.5446 A^-1 at 7 A) and the smallest 2,3,5-smooth grid of at
// least L beta/0.5446 points per axis (the spacing of a 7 A, 0.5446 A^-1
// box), at least 8.
bool smooth235(int k) {
  for (int f : {2, 3, 5})
    while (k % f == 0) k /= f;
  return k == 1;
}

void box_settings(Request& r) {
  if (r.box <= 0.0) return;
  if (!(r.cutoff > 0.0)) r.cutoff = std::min(7.0, 0.5 * r.box - 1e-6);
  if (!(r.beta > 0.0)) r.beta = 3.8122 / r.cutoff;
  if (r.grid <= 0) {
    int k = std::max(8, (int)std::ceil(r.box * r.beta / 0.5446 - 1e-9));
    while (!smooth235(k)) ++k;
    r.grid = k;
  }
}

// Upper estimate of the device bytes of a context solving r (buffers per
// atom, per pair of the lists with their float64/mixed tensors, PME grids),
// used to admit a request that needs a new context. An isolated cluster
// holds up to ~2.8 KB per atom: the all-pairs kernels' column-slice partial
// sums (kClusterMaxSlices x 32 B), the B-spline buffers every context
// allocates (~1 KB), the atom records and the solver vectors.
long long estimate_bytes(const Request& r, int precision) {
  const long long n = r.n;
  if (r.box <= 0.0) return n * 3072 + (16LL << 20);
  const double density = (double)n / (r.box * r.box * r.box);
  const long long half = (long long)(n * 2.0 * M_PI / 3.0 * r.cutoff * r.cutoff * r.cutoff * density) + 1024;
  const long long per_pair = precision == AMP_MIXED ? 4 * (4 + 4 + 4) + 2 * 24 + 24 + 24 : 4 * (4 + 4 + 4) + 2 * 16 + 48;
  const long long K = r.grid, ng = K * K * K, nh = K * K * (K / 2 + 1);
  const long long grids = ng * (8 * 4 + 8 + 4 * 3) + nh * (16 * 3 + 8 * 3);
  return (n * 2048 + half * per_pair) * 5 / 4 + grids + (16LL << 20);
}

double seconds(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Host side of the batched engine: arena, request slots, the work-item list,
// pinned staging for uploads, status reads and results.
struct BatchEngine {
  int max_atoms = 0, max_reqs = 0, max_tiles = 0, n_sm = 1;
  cudaStream_t st = nullptr;
  batch::Arena A{};
  std::vector<void*> dev;  // every device allocation
  int2* d_items = nullptr;
  int* d_heads = nullptr;
  float2* d_tab = nullptr;
  int* d_bad = nullptr;
  double* d_in = nullptr;  // inputs of admitted requests (float64 arrays, concatenated)
  int* d_mol = nullptr;
  double* d_res = nullptr;  // finished requests' dipoles, caller order, concatenated
  long long in_cap = 0, mol_cap = 0, res_cap = 0;
  // pinned host staging
  double* h_in = nullptr;
  int* h_mol = nullptr;
  double* h_res = nullptr;
  long long h_in_cap = 0, h_mol_cap = 0, h_res_cap = 0;
  batch::ReqInfo* h_info = nullptr;
  batch::ReqT* h_reqT = nullptr;
  batch::ReqOut* h_out0 = nullptr;
  batch::ReqOut* h_status[2] = {nullptr, nullptr};
  int2* h_items = nullptr;
  cudaEvent_t ev_status[2] = {nullptr, nullptr}, ev_upload = nullptr, ev_res = nullptr;
  bool upload_pending = false, status_pending[2] = {false, false};
  long long status_launch[2] = {0, 0};
  // slots
  std::vector<std::shared_ptr<Request>> slot;
  std::vector<int> slot_off, slot_tiles;
  std::vector<long long> slot_admitted;  // launch index before which the slot's request was uploaded
  std::map<int, int> free_tiles;         // first tile -> length
  int n_items = 0;
  std::atomic<long long> launches{0};    // iterations launched (pairs of launches)
  // results copied out, delivered once ev_res has completed
  std::vector<std::pair<std::shared_ptr<Request>, long long>> res_pending;  // request, offset in h_res
  Clock::time_point t0;

  template <typename T>
  int alloc(T** p, long long count) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (size_t)std::max(1LL, count)) != cudaSuccess) {
      cudaGetLastError();
      return AMP_ERR_OOM;
    }
    dev.push_back(q);
    *p = (T*)q;
    return AMP_OK;
  }
  template <typename T>
  int grow_dev(T** p, long long* cap, long long need) {
    if (need <= *cap) return AMP_OK;
    if (*p) {
      cudaStreamSynchronize(st);
      for (auto& d : dev)
        if (d == (void*)*p) d = nullptr;
      cudaFree(*p);
      *p = nullptr;
    }
    const long long c = need + need / 2;
    int r = alloc(p, c);
    if (!r) *cap = c;
    return r;
  }
  template <typename T>
  int grow_host(T** p, long long* cap, long long need) {
    if (need <= *cap) return AMP_OK;
    if (*p) {
      cudaStreamSynchronize(st);
      cudaFreeHost(*p);
      *p = nullptr;
    }
    const long long c = need + need / 2;
    if (cudaMallocHost((void**)p, sizeof(T) * (size_t)c) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      *cap = 0;
      return AMP_ERR_OOM;
    }
    *cap = c;
    return AMP_OK;
  }

  long long arena_bytes() const {
    const long long a = max_atoms;
    return a * (16 + 8 + 48 + 48 + 16 + 16 + 8 * 32) + (long long)max_tiles * 32 + (long long)max_reqs * 128;
  }

  int create(int atoms, int reqs, int nsm, const std::vector<float2>& tab) {
    max_tiles = (atoms + batch::kRows - 1) / batch::kRows;
    max_atoms = max_tiles * batch::kRows;
    max_reqs = reqs;
    n_sm = nsm;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return AMP_ERR_CUDA;
    for (auto* e : {&ev_status[0], &ev_status[1], &ev_upload, &ev_res})
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return AMP_ERR_CUDA;
    const long long a = max_atoms;
    int r;
    if ((r = alloc(&A.p32, a)) || (r = alloc(&A.tm32, a)) || (r = alloc(&A.mp32, 3 * a)) ||
        (r = alloc(&A.pdf, 3 * a)) || (r = alloc(&A.v32, a)) || (r = alloc(&A.al, a)) || (r = alloc(&A.e0, a)) ||
        (r = alloc(&A.mu, a)) || (r = alloc(&A.r, a)) || (r = alloc(&A.z, a)) || (r = alloc(&A.p, a)) ||
        (r = alloc(&A.q, a)) || (r = alloc(&A.w, a)) || (r = alloc(&A.tmp, a)) ||
        (r = alloc(&A.part_rz, max_tiles)) || (r = alloc(&A.part_zw, max_tiles)) ||
        (r = alloc(&A.partz, max_tiles)) || (r = alloc(&A.parte, max_tiles)) || (r = alloc(&A.info, reqs)) ||
        (r = alloc(&A.reqT, reqs)) || (r = alloc(&A.reqS, reqs)) || (r = alloc(&A.out, reqs)) ||
        (r = alloc(&d_items, max_tiles)) || (r = alloc(&d_heads, 2)) || (r = alloc(&d_tab, (long long)tab.size())) ||
        (r = alloc(&d_bad, 1)))
      return r;
    if (cudaMallocHost((void**)&h_info, sizeof(batch::ReqInfo) * reqs) != cudaSuccess ||
        cudaMallocHost((void**)&h_reqT, sizeof(batch::ReqT) * reqs) != cudaSuccess ||
        cudaMallocHost((void**)&h_out0, sizeof(batch::ReqOut) * reqs) != cudaSuccess ||
        cudaMallocHost((void**)&h_status[0], sizeof(batch::ReqOut) * reqs) != cudaSuccess ||
        cudaMallocHost((void**)&h_status[1], sizeof(batch::ReqOut) * reqs) != cudaSuccess ||
        cudaMallocHost((void**)&h_items, sizeof(int2) * max_tiles) != cudaSuccess) {
      cudaGetLastError();
      return AMP_ERR_OOM;
    }
    if (cudaMemsetAsync(d_heads, 0, 2 * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(A.out, 0, sizeof(batch::ReqOut) * reqs, st) != cudaSuccess ||
        cudaMemcpyAsync(d_tab, tab.data(), sizeof(float2) * tab.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return AMP_ERR_CUDA;
    slot.assign(reqs, nullptr);
    slot_off.assign(reqs, 0);
    slot_tiles.assign(reqs, 0);
    slot_admitted.assign(reqs, 0);
    free_tiles.clear();
    free_tiles[0] = max_tiles;
    return AMP_OK;
  }

  void destroy() {
    if (st) cudaStreamSynchronize(st);
    for (void* d : dev)
      if (d) cudaFree(d);
    dev.clear();
    for (void* h : {(void*)h_in, (void*)h_mol, (void*)h_res, (void*)h_info, (void*)h_reqT, (void*)h_out0,
                    (void*)h_status[0], (void*)h_status[1], (void*)h_items})
      if (h) cudaFreeHost(h);
    for (cudaEvent_t e : {ev_status[0], ev_status[1], ev_upload, ev_res})
      if (e) cudaEventDestroy(e);
    if (st) cudaStreamDestroy(st);
    st = nullptr;
  }

  // first fit of `tiles` contiguous tiles; -1 if none
  int take_tiles(int tiles) {
    for (auto it = free_tiles.begin(); it != free_tiles.end(); ++it)
      if (it->second >= tiles) {
        const int start = it->first, len = it->second;
        free_tiles.erase(it);
        if (len > tiles) free_tiles[start + tiles] = len - tiles;
        return start;
      }
    return -1;
  }
  void give_tiles(int start, int tiles) {
    auto it = free_tiles.emplace(start, tiles).first;
    auto nx = std::next(it);
    if (nx != free_tiles.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_tiles.erase(nx);
    }
    if (it != free_tiles.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_tiles.erase(it);
      }
    }
  }
  int free_slot() const {
    for (int k = 0; k < max_reqs; ++k)
      if (!slot[k]) return k;
    return -1;
  }
  bool idle() const {
    for (const auto& r : slot)
      if (r) return false;
    return res_pending.empty();
  }
};

}  // namespace serve
}  // namespace amp

struct amp_server {
  amp_server_config cfg{};
  int device = 0, n_sm = 1;
  amp::serve::Clock::time_point t0;
  std::mutex mtx;
  std::condition_variable cv;       // workers and the batch driver: work or stop
  std::condition_variable cv_done;  // waiters: a request finished
  bool stop = false;
  std::deque<std::shared_ptr<amp::serve::Request>> batch_q, work_q;
  std::unordered_map<long long, std::shared_ptr<amp::serve::Request>> reqs;
  long long next_ticket = 0, submitted = 0, done = 0, failed = 0;
  int running_workers = 0, running_batch = 0;
  // context pool: grid size (-1: clusters) -> idle contexts; bytes of every context
  std::multimap<int, amp_ctx*> idle_ctx;
  std::unordered_map<amp_ctx*, long long> ctx_bytes;
  long long ctx_total = 0, reserved = 0;  // bytes of the contexts; reservations for contexts being made
  // resident dipoles of keyed requests (device, caller order), least recently used first
  struct Resident {
    std::string key;
    double* d = nullptr;
    int n = 0;
  };
  std::list<Resident> resident;
  long long resident_total = 0;
  amp::serve::BatchEngine eng;
  bool have_engine = false;
  long long arena_bytes = 0;
  std::vector<std::thread> threads;
  // the workers' streams: owned by the server, destroyed after the pooled
  // contexts (which stay bound to the stream of their last request)
  std::vector<cudaStream_t> worker_streams;
};

namespace amp {
namespace serve {

void finish(amp_server* s, const std::shared_ptr<Request>& r) {  // with s->mtx held
  r->done = true;
  r->res.t_done = seconds(s->t0);
  if (r->res.status == AMP_OK)
    s->done++;
  else
    s->failed++;
  s->cv_done.notify_all();
}

void fail_request(Request& r, int code, const char* msg) {
  r.res.status = code;
  std::snprintf(r.res.error, sizeof(r.res.error), "%s", msg);
}

// ---------------------------------------------------------------- context workers

// An idle context for r's grid size, or a new one when the budget allows (an
// idle context of another size is destroyed to make room); waits while
// neither is possible. Returns null (and fails r) if r can never fit.
amp_ctx* acquire_context(amp_server* s, Request& r, cudaStream_t st, long long* reservation) {
  const int key = r.box > 0.0 ? r.grid : -1;
  std::unique_lock<std::mutex> lk(s->mtx);
  *reservation = 0;
  while (true) {
    auto it = s->idle_ctx.find(key);
    if (it != s->idle_ctx.end()) {
      amp_ctx* c = it->second;
      s->idle_ctx.erase(it);
      return c;
    }
    const long long est = estimate_bytes(r, s->cfg.precision);
    if (est + s->arena_bytes > s->cfg.mem_budget_bytes) {
      fail_request(r, AMP_ERR_OOM, "request larger than the server's memory budget");
      return nullptr;
    }
    if (s->ctx_total + s->reserved + s->resident_total + s->arena_bytes + est <= s->cfg.mem_budget_bytes) {
      s->reserved += est;
      *reservation = est;
      break;
    }
    if (!s->idle_ctx.empty()) {  // make room: the least useful idle context goes
      auto victim = s->idle_ctx.begin();
      amp_ctx* c = victim->second;
      s->idle_ctx.erase(victim);
      s->ctx_total -= s->ctx_bytes[c];
      s->ctx_bytes.erase(c);
      lk.unlock();
      amp_destroy(c);
      lk.lock();
      continue;
    }
    if (!s->resident.empty()) {  // then the resident dipoles
      auto& res = s->resident.front();
      s->resident_total -= (long long)res.n * 3 * sizeof(double);
      cudaFree(res.d);
      s->resident.pop_front();
      continue;
    }
    s->cv.wait(lk);  // a context will come back
  }
  lk.unlock();
  amp_config cfg{};
  cfg.box = r.box > 0.0 ? r.box : 0.0;
  cfg.cutoff = r.cutoff;
  cfg.ewald_beta = r.beta;
  cfg.pme_grid = r.grid > 0 ? r.grid : 8;
  cfg.pme_order = 5;
  cfg.tol_debye = s->cfg.tol_debye;
  cfg.max_iter = s->cfg.max_iter;
  cfg.precision = s->cfg.precision;
  amp_ctx* c = nullptr;
  if (amp_create(&c, &cfg, st) != AMP_OK) {
    std::lock_guard<std::mutex> g(s->mtx);
    s->reserved -= *reservation;
    *reservation = 0;
    fail_request(r, AMP_ERR_CUDA, "amp_create failed");
    return nullptr;
  }
  return c;
}

void release_context(amp_server* s, amp_ctx* c, Request& r, long long reservation, bool healthy) {
  std::lock_guard<std::mutex> g(s->mtx);
  s->reserved -= reservation;
  auto it = s->ctx_bytes.find(c);
  const long long before = it == s->ctx_bytes.end() ? 0 : it->second;
  if (!healthy) {
    s->ctx_total -= before;
    s->ctx_bytes.erase(c);
    amp_destroy(c);
  } else {
    s->ctx_total += c->bytes - before;
    s->ctx_bytes[c] = c->bytes;
    s->idle_ctx.emplace(r.box > 0.0 ? r.grid : -1, c);
  }
  s->cv.notify_all();
}

struct WorkerBuffers {
  double* d = nullptr;  // xyz, q, dip, quad, alpha, thole, E0, mu (caller order)
  int* mol = nullptr;
  long long cap = 0;
  void free_all() {
    if (d) cudaFree(d);
    if (mol) cudaFree(mol);
    d = nullptr;
    mol = nullptr;
    cap = 0;
  }
  int ensure(int n) {
    if (n <= cap) return AMP_OK;
    free_all();
    const long long c = (long long)n + n / 2;
    if (cudaMalloc((void**)&d, sizeof(double) * 21 * c) != cudaSuccess ||
        cudaMalloc((void**)&mol, sizeof(int) * c) != cudaSuccess) {
      cudaGetLastError();
      free_all();
      return AMP_ERR_OOM;
    }
    cap = c;
    return AMP_OK;
  }
};

void run_on_context(amp_server* s, Request& r, cudaStream_t st, WorkerBuffers& wb) {
  const int n = r.n;
  long long reservation = 0;
  amp_ctx* c = acquire_context(s, r, st, &reservation);
  if (!c) return;
  r.res.t_start = seconds(s->t0);
  ctx_bind_stream(c, st);
  bool healthy = true;
  int code = wb.ensure(n);
  if (!code) {
    amp_config cfg = c->cfg;
    if (r.box > 0.0) {
      cfg.box = r.box;
      cfg.cutoff = r.cutoff;
      cfg.ewald_beta = r.beta;
      code = amp_reconfigure(c, &cfg);
    }
  }
  double* xyz = wb.d;
  double *q = xyz + 3LL * wb.cap, *dip = q + wb.cap, *quad = dip + 3LL * wb.cap, *alpha = quad + 6LL * wb.cap;
  double *thole = alpha + wb.cap, *E0 = thole + wb.cap, *mu = E0 + 3LL * wb.cap;
  if (!code) {
    const std::pair<double*, const std::vector<double>*> up[] = {
        {xyz, &r.xyz}, {q, &r.q}, {dip, &r.dip}, {quad, &r.quad}, {alpha, &r.alpha}, {thole, &r.thole}};
    for (const auto& u : up)
      if (cudaMemcpyAsync(u.first, u.second->data(), sizeof(double) * u.second->size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        code = AMP_ERR_CUDA;
    if (cudaMemcpyAsync(wb.mol, r.mol.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
      code = AMP_ERR_CUDA;
  }
  if (!code) code = amp_set_system(c, n, xyz, q, dip, quad, alpha, thole, wb.mol);
  if (!code) code = amp_permanent_field(c, E0);
  int use_guess = 0;
  if (!code && !r.key.empty()) {
    std::lock_guard<std::mutex> g(s->mtx);
    for (auto it = s->resident.begin(); it != s->resident.end(); ++it)
      if (it->key == r.key && it->n == n) {
        cudaMemcpyAsync(mu, it->d, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st);
        s->resident.splice(s->resident.end(), s->resident, it);  // most recently used
        use_guess = 1;
        break;
      }
  }
  int iters = 0;
  double rms = 0.0, U = 0.0;
  if (!code) {
    code = amp_solve_induced(c, E0, mu, use_guess, &iters, &rms);
    if (code == AMP_OK || code == AMP_ERR_NOT_CONVERGED) {
      const int e = amp_polarization_energy(c, mu, E0, &U);
      if (e) code = e;
    }
  }
  if (code == AMP_OK || code == AMP_ERR_NOT_CONVERGED) {
    r.mu.resize(3LL * n);
    if (cudaMemcpyAsync(r.mu.data(), mu, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      code = AMP_ERR_CUDA;
  }
  if (code == AMP_OK && !r.key.empty()) {  // keep the dipoles for the next request of this key
    const long long bytes = 3LL * n * sizeof(double);
    std::lock_guard<std::mutex> g(s->mtx);
    for (auto it = s->resident.begin(); it != s->resident.end(); ++it)
      if (it->key == r.key) {
        s->resident_total -= 3LL * it->n * sizeof(double);
        cudaFree(it->d);
        s->resident.erase(it);
        break;
      }
    while (!s->resident.empty() && s->resident_total + bytes > s->cfg.resident_bytes) {
      s->resident_total -= 3LL * s->resident.front().n * sizeof(double);
      cudaFree(s->resident.front().d);
      s->resident.pop_front();
    }
    double* d = nullptr;
    if (bytes <= s->cfg.resident_bytes && cudaMalloc((void**)&d, bytes) == cudaSuccess) {
      cudaMemcpyAsync(d, mu, bytes, cudaMemcpyDeviceToDevice, st);
      cudaStreamSynchronize(st);
      s->resident.push_back({r.key, d, n});
      s->resident_total += bytes;
    } else {
      cudaGetLastError();
    }
  }
  r.res.iters = iters;
  r.res.rms_debye = rms;
  r.res.energy = U;
  r.res.path = 1;
  r.res.warm_start = use_guess;
  r.res.status = code;
  if (code) {
    std::snprintf(r.res.error, sizeof(r.res.error), "%s", amp_last_error(c));
    if (code == AMP_ERR_CUDA) healthy = false;
  }
  release_context(s, c, r, reservation, healthy);
}

void worker_main(amp_server* s, cudaStream_t st) {
  cudaSetDevice(s->device);
  WorkerBuffers wb;
  while (true) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mtx);
      s->cv.wait(lk, [&] { return s->stop || !s->work_q.empty(); });
      if (s->work_q.empty()) break;  // stopping, nothing left
      r = s->work_q.front();
      s->work_q.pop_front();
      s->running_workers++;
    }
    run_on_context(s, *r, st, wb);
    std::lock_guard<std::mutex> g(s->mtx);
    s->running_workers--;
    finish(s, r);
  }
  cudaStreamSynchronize(st);
  wb.free_all();
}

}  // namespace serve
}  // namespace amp

namespace amp {
namespace serve {

// ---------------------------------------------------------------- batch driver

// Requests from the queue into free slots and tiles (in arrival order; the
// first one that does not fit waits), their inputs uploaded and turned into
// arena records, their slot records initialised. Returns how many joined (or
// a negative error code).
int batch_admit(amp_server* s, BatchEngine& e) {
  std::vector<std::shared_ptr<Request>> in;
  std::vector<int> slots, offs;
  {
    std::lock_guard<std::mutex> g(s->mtx);
    while (!s->batch_q.empty()) {
      const auto& r = s->batch_q.front();
      const int k = e.free_slot();
      const int tiles = (r->n + batch::kRows - 1) / batch::kRows;
      if (k < 0) break;
      const int t = e.take_tiles(tiles);
      if (t < 0) break;
      e.slot[k] = r;  // reserved (the request is not in flight before its upload)
      e.slot_off[k] = t;
      e.slot_tiles[k] = tiles;
      in.push_back(r);
      slots.push_back(k);
      offs.push_back(t * batch::kRows);
      s->batch_q.pop_front();
      s->running_batch++;
    }
  }
  if (in.empty()) return 0;
  long long nd = 0, nm = 0;
  for (const auto& r : in) {
    nd += 15LL * r->n;
    nm += r->n;
  }
  // the pinned staging of the last upload must have been read
  if (e.upload_pending) cudaEventSynchronize(e.ev_upload);
  int rc;
  if ((rc = e.grow_host(&e.h_in, &e.h_in_cap, nd)) || (rc = e.grow_host(&e.h_mol, &e.h_mol_cap, nm)) ||
      (rc = e.grow_dev(&e.d_in, &e.in_cap, nd)) || (rc = e.grow_dev(&e.d_mol, &e.mol_cap, nm))) {
    std::lock_guard<std::mutex> g(s->mtx);
    for (size_t k = 0; k < in.size(); ++k) {  // these requests fail alone
      fail_request(*in[k], rc, "no memory to stage the request");
      finish(s, in[k]);
      e.give_tiles(e.slot_off[slots[k]], e.slot_tiles[slots[k]]);
      e.slot[slots[k]] = nullptr;
      s->running_batch--;
    }
    return rc;
  }
  long long od = 0, om = 0;
  std::vector<long long> od_of, om_of;
  for (const auto& r : in) {
    od_of.push_back(od);
    om_of.push_back(om);
    const std::vector<double>* parts[] = {&r->xyz, &r->q, &r->dip, &r->quad, &r->alpha, &r->thole};
    for (const auto* v : parts) {
      std::memcpy(e.h_in + od, v->data(), sizeof(double) * v->size());
      od += (long long)v->size();
    }
    std::memcpy(e.h_mol + om, r->mol.data(), sizeof(int) * r->n);
    om += r->n;
  }
  cudaMemcpyAsync(e.d_in, e.h_in, sizeof(double) * od, cudaMemcpyHostToDevice, e.st);
  cudaMemcpyAsync(e.d_mol, e.h_mol, sizeof(int) * om, cudaMemcpyHostToDevice, e.st);
  const double t_start = seconds(s->t0);
  for (size_t k = 0; k < in.size(); ++k) {
    const Request& r = *in[k];
    const int n = r.n, sl = slots[k];
    const double* base = e.d_in + od_of[k];
    batch::k_batch_records<<<amp_blocks(n, 128), 128, 0, e.st>>>(
        offs[k], n, base, base + 3LL * n, base + 4LL * n, base + 7LL * n, base + 13LL * n, base + 14LL * n,
        e.d_mol + om_of[k], e.A, e.d_bad);
    batch::ReqInfo& info = e.h_info[sl];
    info.off = offs[k];
    info.n = n;
    info.tile0 = e.slot_off[sl];
    info.ntiles = e.slot_tiles[sl];
    info.tol = s->cfg.tol_debye;
    info.max_iter = s->cfg.max_iter;
    info.pad = 0;
    e.h_reqT[sl] = batch::ReqT{batch::K_E0, 0, 1, 0, 0.0, 0.0};
    e.h_out0[sl] = batch::ReqOut{0, 0, 0.0, 0.0};
    cudaMemcpyAsync(e.A.info + sl, e.h_info + sl, sizeof(batch::ReqInfo), cudaMemcpyHostToDevice, e.st);
    cudaMemcpyAsync(e.A.reqT + sl, e.h_reqT + sl, sizeof(batch::ReqT), cudaMemcpyHostToDevice, e.st);
    cudaMemcpyAsync(e.A.out + sl, e.h_out0 + sl, sizeof(batch::ReqOut), cudaMemcpyHostToDevice, e.st);
    e.slot_admitted[sl] = e.launches;
    in[k]->res.t_start = t_start;
  }
  return (int)in.size();
}

// The work items of the requests in flight, larger requests first (their
// items are the longest), uploaded for the next launches.
void batch_items(BatchEngine& e) {
  if (e.upload_pending) cudaEventSynchronize(e.ev_upload);  // h_items of the last upload has been read
  std::vector<int> order;
  for (int k = 0; k < e.max_reqs; ++k)
    if (e.slot[k]) order.push_back(k);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return e.slot[a]->n > e.slot[b]->n; });
  int m = 0;
  for (int k : order)
    for (int t = 0; t < e.slot_tiles[k]; ++t) e.h_items[m++] = make_int2(k, t);
  e.n_items = m;
  if (m) cudaMemcpyAsync(e.d_items, e.h_items, sizeof(int2) * m, cudaMemcpyHostToDevice, e.st);
  cudaEventRecord(e.ev_upload, e.st);
  e.upload_pending = true;
}

// Results whose copy has completed go to their requests.
void batch_deliver(amp_server* s, BatchEngine& e, bool wait) {
  if (e.res_pending.empty()) return;
  if (!wait && cudaEventQuery(e.ev_res) == cudaErrorNotReady) return;
  cudaEventSynchronize(e.ev_res);
  std::lock_guard<std::mutex> g(s->mtx);
  for (auto& p : e.res_pending) {
    Request& r = *p.first;
    r.mu.assign(e.h_res + p.second, e.h_res + p.second + 3LL * r.n);
    finish(s, p.first);
  }
  e.res_pending.clear();
}

// Requests that ended in launch `launch` (end records read into h): their
// dipoles are copied out, their slots and tiles freed.
int batch_retire(amp_server* s, BatchEngine& e, const batch::ReqOut* h, long long launch) {
  std::vector<int> fin;
  for (int k = 0; k < e.max_reqs; ++k)
    if (e.slot[k] && e.slot_admitted[k] <= launch && h[k].status != 0) fin.push_back(k);
  if (fin.empty()) return 0;
  batch_deliver(s, e, true);  // h_res is free again
  long long need = 0;
  for (int k : fin) need += 3LL * e.slot[k]->n;
  if (e.grow_dev(&e.d_res, &e.res_cap, need) || e.grow_host(&e.h_res, &e.h_res_cap, need)) {
    std::lock_guard<std::mutex> g(s->mtx);
    for (int k : fin) {
      fail_request(*e.slot[k], AMP_ERR_OOM, "no memory for the result");
      finish(s, e.slot[k]);
      e.give_tiles(e.slot_off[k], e.slot_tiles[k]);
      e.slot[k] = nullptr;
      s->running_batch--;
    }
    return (int)fin.size();
  }
  long long o = 0;
  for (int k : fin) {
    Request& r = *e.slot[k];
    const batch::ReqOut& out = h[k];
    batch::k_batch_result<<<amp_blocks(r.n, 128), 128, 0, e.st>>>(e.slot_off[k] * batch::kRows, r.n, e.A.mu,
                                                                  e.d_res + o);
    r.res.status = out.status == 1 ? AMP_OK : AMP_ERR_NOT_CONVERGED;
    if (out.status == 2) std::snprintf(r.res.error, sizeof(r.res.error), "PCG not converged after %d iterations", out.iters);
    if (out.status == 3) std::snprintf(r.res.error, sizeof(r.res.error), "PCG breakdown: p.Ap <= 0");
    r.res.iters = out.iters;
    r.res.rms_debye = out.rms;
    r.res.energy = out.U;
    r.res.path = 0;
    e.res_pending.emplace_back(e.slot[k], o);
    o += 3LL * r.n;
    e.give_tiles(e.slot_off[k], e.slot_tiles[k]);
    e.slot[k] = nullptr;
  }
  cudaMemcpyAsync(e.h_res, e.d_res, sizeof(double) * o, cudaMemcpyDeviceToHost, e.st);
  cudaEventRecord(e.ev_res, e.st);
  std::lock_guard<std::mutex> g(s->mtx);
  s->running_batch -= (int)fin.size();
  return (int)fin.size();
}

// The driver: admit, launch one iteration of everything in flight, read the
// end records of the iteration before (the GPU has this one queued
// meanwhile), retire, deliver; sleep when there is nothing to do.
void batch_main(amp_server* s) {
  cudaSetDevice(s->device);
  BatchEngine& e = s->eng;
  const int grid_cap = 8 * s->n_sm;
  bool items_dirty = false;
  int cur = 0;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s->mtx);
      const bool busy = s->running_batch > 0 || !e.res_pending.empty() || e.status_pending[0] || e.status_pending[1];
      if (!busy) s->cv.wait(lk, [&] { return s->stop || !s->batch_q.empty(); });
      if (s->stop && s->batch_q.empty() && !busy) break;
    }
    if (batch_admit(s, e) > 0) items_dirty = true;
    if (items_dirty) {
      batch_items(e);
      items_dirty = false;
    }
    bool launched = false;
    if (e.n_items > 0) {
      const int grid = std::min(e.n_items, grid_cap);
      batch::k_batch_pairs<<<grid, batch::kThreads, 0, e.st>>>(e.A, e.n_items, e.d_items, e.d_heads, e.d_tab);
      batch::k_batch_vectors<<<grid, batch::kThreads, 0, e.st>>>(e.A, e.n_items, e.d_items, e.d_heads);
      cudaMemcpyAsync(e.h_status[cur], e.A.out, sizeof(batch::ReqOut) * e.max_reqs, cudaMemcpyDeviceToHost, e.st);
      cudaEventRecord(e.ev_status[cur], e.st);
      e.status_pending[cur] = true;
      e.status_launch[cur] = e.launches;
      e.launches++;
      launched = true;
    }
    // the end records of the iteration before are read while this one runs;
    // with nothing launched, those of this round's buffer too
    for (int b : {cur ^ 1, cur}) {
      if (b == cur && launched) continue;
      if (!e.status_pending[b]) continue;
      cudaEventSynchronize(e.ev_status[b]);
      e.status_pending[b] = false;
      if (batch_retire(s, e, e.h_status[b], e.status_launch[b]) > 0) items_dirty = true;
    }
    batch_deliver(s, e, !launched);
    cur ^= 1;
  }
  batch_deliver(s, e, true);
}

bool valid_inputs(int n, const double* alpha) {
  for (int i = 0; i < n; ++i)
    if (!(alpha[i] > 0.0)) return false;
  return true;
}

}  // namespace serve
}  // namespace amp

using namespace amp::serve;

extern "C" {

int amp_server_create(amp_server** out, const amp_server_config* cfg, int device) {
  if (!out) return AMP_ERR_ARG;
  *out = nullptr;
  if (!cfg || cfg->n_workers < 1 || cfg->mem_budget_bytes <= 0 || !(cfg->tol_debye > 0.0) || cfg->max_iter < 1 ||
      (cfg->precision != AMP_FP64 && cfg->precision != AMP_MIXED) || cfg->batch_max_atoms < 0 ||
      (cfg->batch_max_atoms > 0 &&
       (cfg->batch_arena_atoms < cfg->batch_max_atoms || cfg->batch_max_requests < 1)) ||
      cfg->resident_bytes < 0)
    return AMP_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return AMP_ERR_CUDA;
  }
  amp_server* s = new (std::nothrow) amp_server();
  if (!s) return AMP_ERR_OOM;
  s->cfg = *cfg;
  s->device = device;
  s->t0 = Clock::now();
  if (cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || s->n_sm < 1)
    s->n_sm = 1;
  if (cfg->batch_max_atoms > 0) {
    std::vector<float2> tab;
    amp::dfm_host_table(tab);
    const int r = s->eng.create(cfg->batch_arena_atoms, cfg->batch_max_requests, s->n_sm, tab);
    if (r) {
      s->eng.destroy();
      delete s;
      return r;
    }
    s->have_engine = true;
    s->arena_bytes = s->eng.arena_bytes();
    if (s->arena_bytes > cfg->mem_budget_bytes) {
      s->eng.destroy();
      delete s;
      return AMP_ERR_ARG;
    }
  }
  for (int k = 0; k < cfg->n_workers; ++k) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (cudaStream_t w : s->worker_streams) cudaStreamDestroy(w);
      if (s->have_engine) s->eng.destroy();
      delete s;
      return AMP_ERR_CUDA;
    }
    s->worker_streams.push_back(st);
  }
  for (int k = 0; k < cfg->n_workers; ++k) s->threads.emplace_back(worker_main, s, s->worker_streams[k]);
  if (s->have_engine) s->threads.emplace_back(batch_main, s);
  *out = s;
  return AMP_OK;
}

int amp_server_submit(amp_server* s, int n, double box, double cutoff, double beta, int grid, const double* xyz,
                      const double* q, const double* dip, const double* quad, const double* alpha,
                      const double* thole, const int* mol, const char* key, long long* ticket) {
  if (!s || !ticket || n < 2 || !xyz || !q || !dip || !quad || !alpha || !thole || !mol || !(box >= 0.0))
    return AMP_ERR_ARG;
  auto r = std::make_shared<Request>();
  r->n = n;
  r->box = box;
  r->cutoff = cutoff;
  r->beta = beta;
  r->grid = grid;
  r->xyz.assign(xyz, xyz + 3LL * n);
  r->q.assign(q, q + n);
  r->dip.assign(dip, dip + 3LL * n);
  r->quad.assign(quad, quad + 6LL * n);
  r->alpha.assign(alpha, alpha + n);
  r->thole.assign(thole, thole + n);
  r->mol.assign(mol, mol + n);
  if (key) r->key = key;
  box_settings(*r);
  std::lock_guard<std::mutex> g(s->mtx);
  if (s->stop) return AMP_ERR_STATE;
  r->ticket = s->next_ticket++;
  r->res.t_submit = seconds(s->t0);
  *ticket = r->ticket;
  s->reqs[r->ticket] = r;
  s->submitted++;
  if (!valid_inputs(n, alpha)) {
    fail_request(*r, AMP_ERR_ARG, "alpha must be > 0 for every site");
    finish(s, r);
    return AMP_OK;
  }
  if (box > 0.0 && !(2.0 * r->cutoff < box)) {
    fail_request(*r, AMP_ERR_ARG, "cutoff must be below box/2");
    finish(s, r);
    return AMP_OK;
  }
  if (s->have_engine && box == 0.0 && n <= s->cfg.batch_max_atoms && r->key.empty())
    s->batch_q.push_back(r);
  else
    s->work_q.push_back(r);
  s->cv.notify_all();
  return AMP_OK;
}

static int take_result(amp_server* s, long long ticket, double* mu, amp_server_result* res) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return AMP_ERR_ARG;
  const auto& r = it->second;
  if (!r->done) return AMP_PENDING;
  if (mu && !r->mu.empty()) std::memcpy(mu, r->mu.data(), sizeof(double) * r->mu.size());
  if (res) *res = r->res;
  const int st = r->res.status;
  s->reqs.erase(it);
  return st;
}

int amp_server_poll(amp_server* s, long long ticket, double* mu, amp_server_result* res) {
  if (!s) return AMP_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mtx);
  return take_result(s, ticket, mu, res);
}

int amp_server_wait(amp_server* s, long long ticket, double timeout_s, double* mu, amp_server_result* res) {
  if (!s) return AMP_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mtx);
  auto ready = [&] {
    auto it = s->reqs.find(ticket);
    return it == s->reqs.end() || it->second->done;
  };
  if (timeout_s < 0.0)
    s->cv_done.wait(lk, ready);
  else
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
  return take_result(s, ticket, mu, res);
}

int amp_server_stats(amp_server* s, amp_server_counters* out) {
  if (!s || !out) return AMP_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mtx);
  out->submitted = s->submitted;
  out->done = s->done;
  out->failed = s->failed;
  out->queued = (int)(s->batch_q.size() + s->work_q.size());
  out->running_batch = s->running_batch;
  out->running_workers = s->running_workers;
  out->contexts = (int)s->ctx_bytes.size();
  out->bytes_in_use = s->ctx_total + s->reserved + s->resident_total + s->arena_bytes;
  out->budget = s->cfg.mem_budget_bytes;
  out->batch_launches = 2 * s->eng.launches.load();
  return AMP_OK;
}

void amp_server_destroy(amp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mtx);
    s->stop = true;
    s->cv.notify_all();
  }
  for (auto& t : s->threads) t.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->idle_ctx) amp_destroy(kv.second);
  for (auto& r : s->resident) cudaFree(r.d);
  if (s->have_engine) s->eng.destroy();
  for (cudaStream_t st : s->worker_streams) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
