// Serving: continuous batching of single OCP requests over the persistent
// solver kernel (include/to.h: toserver_create, tosubmit, topoll).
//
// Per problem the server owns a pool of seats (one instance workspace each,
// sized from the HBM budget), a descriptor ring, a "tail" counter, per-seat
// completion flags and results, all but the seats in pinned, device-mapped
// host memory.  tosubmit admits a request only into a free seat, writes its
// descriptor (x0 inline), publishes it by advancing tail and makes sure a
// solver kernel runs on the problem's stream.  The running kernel's idle
// groups claim published requests at every outer iteration, so requests that
// arrive while others are mid-solve start at once and share the GPU with
// them.  A kernel whose groups are all idle polls for a bounded time and
// leaves; the next submit (or poll) launches a new one.  topoll returns a
// request's results once its seat's flag carries the request's ring index.
//
// A launch that has had no group solving for a while closes: it latches a
// flag that stops all its claims and drains.  The host keeps two launch
// slots per problem (a stream, an event and a control block each), so a
// successor can start while the closing launch finishes its last solves.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "handles.h"

using namespace to;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Lane {
  to_problem p = nullptr;
  to_batch b = nullptr;
  int seats = 0;
  cudaStream_t stream[2] = {nullptr, nullptr}, copy = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool launched[2] = {false, false};
  int cur = 0;               // launch slot of the newest launch
  double share = 1.0;        // fraction of the resident CTAs this problem's kernel takes
  int* ctl = nullptr;        // device: two control blocks of two ints
  int* closing_h = nullptr;  // host-mapped closing latches, one per slot
  int* closing_d = nullptr;
  int ring_size = 0;
  ServeDesc* ring_h = nullptr;
  ServeDesc* ring_d = nullptr;
  unsigned* tail_h = nullptr;
  unsigned* tail_d = nullptr;
  unsigned* done_h = nullptr;
  unsigned* done_d = nullptr;
  int* stop_h = nullptr;
  int* stop_d = nullptr;
  double* J_h = nullptr;
  double* J_d = nullptr;
  int* it_h = nullptr;
  int* it_d = nullptr;
  int* st_h = nullptr;
  int* st_d = nullptr;
  unsigned* head = nullptr;
  int* seat_T = nullptr;
  long long* seat_toff = nullptr;
  double* gX = nullptr;
  double* gU = nullptr;
  double* own_J = nullptr;   // the batch's own result buffers, put back before it is freed
  int* own_it = nullptr;
  int* own_st = nullptr;
  std::vector<int> free_seats;
  unsigned next_q = 0;
};

struct Req {
  int lane, seat;
  unsigned seq;
  double t_submit;
};

}  // namespace

struct to_server_s {
  std::vector<Lane> lanes;
  to_solver_opts opts;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_id = 1;
  long long completed = 0;
  size_t bytes = 0;
  std::mutex mu;
};

#define SV_CK(x)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) return to_fail(TO_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
static cudaError_t mapped(T** host, T** dev, size_t count) {
  cudaError_t e = cudaHostAlloc((void**)host, std::max<size_t>(count, 1) * sizeof(T), cudaHostAllocMapped);
  if (e != cudaSuccess) return e;
  std::memset(*host, 0, std::max<size_t>(count, 1) * sizeof(T));
  return cudaHostGetDevicePointer((void**)dev, *host, 0);
}

static bool kernel_running(Lane& L, int k) { return L.launched[k] && cudaEventQuery(L.ev[k]) == cudaErrorNotReady; }

// make sure a launch that still claims requests runs for the lane
static int pump(to_server s, Lane& L) {
  const int c = L.cur;
  const bool run_c = kernel_running(L, c);
  if (run_c && !reinterpret_cast<volatile int*>(L.closing_h)[c]) return TO_OK;
  const int k = run_c ? c ^ 1 : c;
  if (kernel_running(L, k)) return TO_OK;   // both slots still draining: a later poll retries
  // slot k is free: reset its control block (stream-ordered before the kernel)
  reinterpret_cast<volatile int*>(L.closing_h)[k] = 0;
  SV_CK(cudaMemsetAsync(L.ctl + 2 * k, 0, 2 * sizeof(int), L.stream[k]));
  ServeArgs sa{};
  sa.ring = L.ring_d;
  sa.ring_size = L.ring_size;
  sa.tail = L.tail_d;
  sa.head = L.head;
  sa.done = L.done_d;
  sa.stop = L.stop_d;
  sa.seat_T = L.seat_T;
  sa.ctl = L.ctl + 2 * k;
  sa.closing = L.closing_d + k;
  sa.idle_polls = 500;          // about 1 ms with no group solving before the launch closes
  sa.grid_frac = L.share;
  int rc = to_launch_core(L.b, L.seats, nullptr, nullptr, nullptr, nullptr, &s->opts, L.stream[k], &sa);
  if (rc) return rc;
  SV_CK(cudaEventRecord(L.ev[k], L.stream[k]));
  L.launched[k] = true;
  L.cur = k;
  return TO_OK;
}

static void free_lane(Lane& L) {
  if (L.stop_h) *reinterpret_cast<volatile int*>(L.stop_h) = 1;
  for (cudaStream_t st : L.stream)
    if (st) cudaStreamSynchronize(st);
  if (L.copy) cudaStreamSynchronize(L.copy);
  if (L.b) {
    if (L.own_J) {
      L.b->J = L.own_J;
      L.b->iters = L.own_it;
      L.b->status = L.own_st;
    }
    tofree_batch(L.b);
  }
  void* hostp[] = {L.ring_h, L.tail_h, L.done_h, L.stop_h, L.J_h, L.it_h, L.st_h, L.closing_h};
  for (void* q : hostp)
    if (q) cudaFreeHost(q);
  void* devp[] = {L.head, L.seat_T, L.seat_toff, L.gX, L.gU, L.ctl};
  for (void* q : devp)
    if (q) cudaFree(q);
  for (int k = 0; k < 2; ++k) {
    if (L.ev[k]) cudaEventDestroy(L.ev[k]);
    if (L.stream[k]) cudaStreamDestroy(L.stream[k]);
  }
  if (L.copy) cudaStreamDestroy(L.copy);
}

int toserver_create(const to_problem* problems, int n_problems, const to_solver_opts* opts, size_t hbm_budget_bytes,
                    to_server* out) {
  if (!problems || n_problems < 1 || !out) return to_fail(TO_ERR_ARG, "toserver_create: bad arguments");
  *out = nullptr;
  to_server s = new to_server_s();
  to_default_opts(&s->opts);
  if (opts) s->opts = *opts;
  s->opts.forced_alpha = nullptr;
  s->opts.want_vx = 0;
  s->opts.profile_phases = 0;
  const size_t budget = hbm_budget_bytes ? hbm_budget_bytes : ((size_t)4 << 30);
  s->lanes.resize(n_problems);
  for (int pi = 0; pi < n_problems; ++pi) {
    Lane& L = s->lanes[pi];
    to_problem p = problems[pi];
    if (!p || p->n > kServeMaxN) {
      toserver_destroy(s);
      return to_fail(TO_ERR_ARG, "toserver_create: bad problem handle");
    }
    L.p = p;
    const int pr = s->opts.prec == TO_FP64 ? 0 : 1;
    const int elem = pr == 0 ? 8 : 4;
    const size_t per_seat = (size_t)(p->T_max + 1) * (kMaxSlots * p->ops->rs[pr] + p->ops->gs[pr] + p->knot_scratch[pr]) * elem +
                            (size_t)(s->opts.max_iter + 1) * 12 + 64;
    L.seats = (int)std::min<size_t>(budget / n_problems / per_seat, 1 << 16);
    if (L.seats < 1) {
      toserver_destroy(s);
      return to_fail(TO_ERR_BUDGET, "toserver_create: the HBM budget does not hold one request workspace");
    }
    to_solver_opts bo = s->opts;
    bo.hbm_budget_bytes = 0;
    int rc = tocreate_batch(p, L.seats, (long long)L.seats * (p->T_max + 1), &bo, &L.b);
    if (rc) {
      toserver_destroy(s);
      return rc;
    }
    L.ring_size = 2 * L.seats;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = mapped(&L.ring_h, &L.ring_d, L.ring_size);
    if (e == cudaSuccess) e = mapped(&L.tail_h, &L.tail_d, 1);
    if (e == cudaSuccess) e = mapped(&L.done_h, &L.done_d, L.seats);
    if (e == cudaSuccess) e = mapped(&L.stop_h, &L.stop_d, 1);
    if (e == cudaSuccess) e = mapped(&L.J_h, &L.J_d, L.seats);
    if (e == cudaSuccess) e = mapped(&L.it_h, &L.it_d, L.seats);
    if (e == cudaSuccess) e = mapped(&L.st_h, &L.st_d, L.seats);
    if (e == cudaSuccess) e = mapped(&L.closing_h, &L.closing_d, 2);
    if (e == cudaSuccess) e = cudaMalloc(&L.ctl, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(L.ctl, 0, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&L.head, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(L.head, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&L.seat_T, sizeof(int) * L.seats);
    if (e == cudaSuccess) e = cudaMalloc(&L.seat_toff, sizeof(long long) * L.seats);
    if (e == cudaSuccess) e = cudaMalloc(&L.gX, sizeof(double) * (p->T_max + 1) * p->n);
    if (e == cudaSuccess) e = cudaMalloc(&L.gU, sizeof(double) * p->T_max * p->m);
    if (e == cudaSuccess) {
      std::vector<long long> toff(L.seats);
      for (int i = 0; i < L.seats; ++i) toff[i] = (long long)i * (p->T_max + 1);
      e = cudaMemcpy(L.seat_toff, toff.data(), sizeof(long long) * L.seats, cudaMemcpyHostToDevice);
    }
    // per-iteration history buffers the kernel writes
    if (e == cudaSuccess) e = cudaMalloc(&L.b->ahist, sizeof(int) * (size_t)L.seats * std::max(s->opts.max_iter, 1));
    if (e == cudaSuccess) e = cudaMalloc(&L.b->Jhist, sizeof(double) * (size_t)L.seats * (s->opts.max_iter + 1));
    if (e == cudaSuccess) e = cudaMemset(L.b->err, 0, sizeof(int));
    for (int k = 0; k < 2; ++k) {
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.stream[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.ev[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      toserver_destroy(s);
      return to_fail(TO_ERR_CUDA, std::string("toserver_create: ") + cudaGetErrorString(e));
    }
    L.b->hist_iter_cap = s->opts.max_iter;
    // the kernel writes results and completion flags straight to host memory
    L.own_J = L.b->J; L.own_it = L.b->iters; L.own_st = L.b->status;
    L.b->J = L.J_d; L.b->iters = L.it_d; L.b->status = L.st_d;
    L.free_seats.resize(L.seats);
    for (int i = 0; i < L.seats; ++i) L.free_seats[i] = L.seats - 1 - i;
    s->bytes += L.b->bytes;
  }
  // Each problem's kernel takes an equal share of the resident CTAs.  (Shares
  // weighted by per-request work measured worse: a heavy problem's closing
  // launch and its successor then hold most of the GPU between them, and the
  // other problems' launches wait for residency.)
  for (int pi = 0; pi < n_problems; ++pi) s->lanes[pi].share = 1.0 / n_problems;
  *out = s;
  return TO_OK;
}

void toserver_destroy(to_server s) {
  if (!s) return;
  for (Lane& L : s->lanes) free_lane(L);
  delete s;
}

int tosubmit(to_server s, int problem, const double* x0, int T, uint64_t* req_id) {
  if (!s || !x0 || !req_id) return to_fail(TO_ERR_ARG, "tosubmit: null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  if (problem < 0 || problem >= (int)s->lanes.size()) return to_fail(TO_ERR_ARG, "tosubmit: bad problem index");
  Lane& L = s->lanes[problem];
  if (T < 1 || T > L.p->T_max) return to_fail(TO_ERR_ARG, "tosubmit: horizon outside [1, T_max]");
  if (L.free_seats.empty()) return to_fail(TO_ERR_BUDGET, "tosubmit: no free seat within the HBM budget; poll and retry");
  const int seat = L.free_seats.back();
  L.free_seats.pop_back();
  const unsigned q = L.next_q++;
  ServeDesc& d = L.ring_h[q % L.ring_size];
  d.seat = seat;
  d.T = T;
  d.seq = q + 1;
  for (int i = 0; i < L.p->n; ++i) d.x0[i] = x0[i];
  reinterpret_cast<volatile unsigned*>(L.done_h)[seat] = 0;
  std::atomic_thread_fence(std::memory_order_seq_cst);   // descriptor before the tail
  *reinterpret_cast<volatile unsigned*>(L.tail_h) = q + 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  const uint64_t id = s->next_id++;
  s->reqs[id] = Req{problem, seat, q + 1, now_ms()};
  *req_id = id;
  return pump(s, L);
}

int topoll(to_server s, uint64_t req_id, double* X, double* U, double* J, int* iters, int* status, double* latency_ms) {
  if (!s) return to_fail(TO_ERR_ARG, "topoll: null server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return to_fail(TO_ERR_ARG, "topoll: unknown request id");
  Req r = it->second;
  Lane& L = s->lanes[r.lane];
  if (reinterpret_cast<volatile unsigned*>(L.done_h)[r.seat] != r.seq) {
    const int rc = pump(s, L);        // a kernel that left just before the request was published
    if (rc) return rc;
    return TO_ERR_NOTREADY;
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  const double t_done = now_ms();
  if (J) *J = reinterpret_cast<volatile double*>(L.J_h)[r.seat];
  if (iters) *iters = reinterpret_cast<volatile int*>(L.it_h)[r.seat];
  if (status) *status = reinterpret_cast<volatile int*>(L.st_h)[r.seat];
  if (X || U) {
    to_problem p = L.p;
    const int pr = L.b->prec == TO_FP64 ? 0 : 1;
    const int NS = std::min(L.b->G, kLsWidth) + 1;
    gather_kernel<<<64, 256, 0, L.copy>>>(1, p->T_max, p->n, p->m, p->ops->rs[pr], p->ops->gs[pr], NS,
                                          pr == 0 ? 8 : 4, L.seat_toff + r.seat, L.seat_T + r.seat,
                                          L.b->slot + r.seat, L.b->traj, L.b->gains, nullptr, X ? L.gX : nullptr,
                                          U ? L.gU : nullptr, nullptr, nullptr, nullptr);
    SV_CK(cudaGetLastError());
    if (X) SV_CK(cudaMemcpyAsync(X, L.gX, sizeof(double) * (p->T_max + 1) * p->n, cudaMemcpyDeviceToHost, L.copy));
    if (U) SV_CK(cudaMemcpyAsync(U, L.gU, sizeof(double) * p->T_max * p->m, cudaMemcpyDeviceToHost, L.copy));
    SV_CK(cudaStreamSynchronize(L.copy));
  }
  if (latency_ms) *latency_ms = t_done - r.t_submit;
  L.free_seats.push_back(r.seat);
  s->reqs.erase(it);
  ++s->completed;
  return TO_OK;
}

int toserver_stats(to_server s, int* seats_total, int* seats_busy, long long* completed, size_t* hbm_bytes) {
  if (!s) return to_fail(TO_ERR_ARG, "toserver_stats: null server");
  std::lock_guard<std::mutex> lock(s->mu);
  int tot = 0, busy = 0;
  for (Lane& L : s->lanes) {
    tot += L.seats;
    busy += L.seats - (int)L.free_seats.size();
  }
  if (seats_total) *seats_total = tot;
  if (seats_busy) *seats_busy = busy;
  if (completed) *completed = s->completed;
  if (hbm_bytes) *hbm_bytes = s->bytes;
  return TO_OK;
}

int toserve_replay(to_server s, int n_req, const double* arrival_s, const int* problem, const int* T,
                   const double* x0, int x0_stride, double* latency_ms, double* J, int* status, double timeout_s) {
  if (!s || n_req < 0 || (n_req > 0 && (!arrival_s || !problem || !T || !x0 || !latency_ms)))
    return to_fail(TO_ERR_ARG, "toserve_replay: bad arguments");
  std::vector<uint64_t> ids(n_req, 0);
  std::vector<char> done(n_req, 0);
  const double t0 = now_ms();
  int next = 0, finished = 0;
  std::vector<int> pending;     // arrived, waiting for a seat (in arrival order)
  size_t scan = 0;
  std::vector<int> active;
  while (finished < n_req) {
    const double t = now_ms() - t0;
    if (t > timeout_s * 1e3) return to_fail(TO_ERR_TIMEOUT, "toserve_replay: trace did not finish in time");
    while (next < n_req && arrival_s[next] * 1e3 <= t) pending.push_back(next++);
    // admit arrived requests while seats are free (oldest first)
    size_t k = 0;
    for (; k < pending.size(); ++k) {
      const int i = pending[k];
      const int rc = tosubmit(s, problem[i], x0 + (size_t)i * x0_stride, T[i], &ids[i]);
      if (rc == TO_ERR_BUDGET) break;
      if (rc) return rc;
      active.push_back(i);
    }
    pending.erase(pending.begin(), pending.begin() + k);
    // poll the active requests
    for (size_t a = 0; a < active.size();) {
      const int i = active[a];
      double lat = 0, Jv = 0;
      int st = 0;
      const int rc = topoll(s, ids[i], nullptr, nullptr, &Jv, nullptr, &st, &lat);
      if (rc == TO_ERR_NOTREADY) { ++a; continue; }
      if (rc) return rc;
      // latency from the scheduled arrival (includes any wait for a seat)
      latency_ms[i] = now_ms() - t0 - arrival_s[i] * 1e3;
      if (J) J[i] = Jv;
      if (status) status[i] = st;
      done[i] = 1;
      ++finished;
      active[a] = active.back();
      active.pop_back();
    }
    (void)scan;
  }
  return TO_OK;
}
