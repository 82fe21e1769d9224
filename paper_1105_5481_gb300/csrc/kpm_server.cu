// Serving loop with continuous batching (kpm_server_*).
//
// Requests (a handle, its parameters and a DOS node count) are queued by
// kpm_server_submit from any thread.  A scheduler thread owns one CUDA stream
// and a device arena of the HBM budget, and runs ticks:
//   1. admission: pending requests, first come first served, are made
//      resident as soon as their device memory (two vector blocks, scaled
//      operator, moment sums and outputs, DOS buffers) fits in the arena;
//   2. advance: small and medium requests, grouped by operator kind and
//      vector width, move up to `steps_per_tick` products together in one
//      batched persistent cluster launch per group (the instance task table is
//      rewritten every tick, so requests that arrived during the previous tick
//      join this one); the tick waits for these launches only.  Large
//      requests (a product moving >= 8 MB) run as full-GPU fused steps on a
//      pool of streams, SOLO_CHUNK_TICKS * steps_per_tick products per
//      enqueue, overlapping with the batched launches and with each other; the
//      scheduler polls an event per large request and enqueues its next chunk
//      once the previous one has finished, so the small requests' ticks are
//      never paced by the large ones;
//   3. retirement: finished requests get their Jackson DOS on the device,
//      their results are copied to the host, their arena memory is released
//      (for a large request only after its last chunk has completed) and
//      their waiters are woken.
// A request's products are split among CTAs by a partition that depends only
// on its own shape (and the server's cluster size), so its moments are the
// same alone and in any mix, however its steps are spread over ticks.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kpm_batch.cuh"

using namespace kpm;

namespace {

// Requests whose product moves at least this many bytes (3 N Rp s_v) run as
// full-GPU fused steps; smaller ones share the batched cluster launches.
constexpr size_t SOLO_STEP_BYTES = size_t(8) << 20;
constexpr int MAX_GROUPS = 1024;
constexpr int SOLO_STREAMS = 4;
constexpr int SOLO_CHUNK_TICKS = 4;
constexpr size_t ALIGN = 256;

size_t al(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocator over one device allocation; freed ranges coalesce.
class Arena {
 public:
  cudaError_t init(size_t bytes) {
    cap_ = al(bytes);
    cudaError_t e = cudaMalloc(&base_, cap_);
    if (e != cudaSuccess) return e;
    free_[0] = cap_;
    return cudaSuccess;
  }
  void destroy() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = al(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* base() const { return (char*)base_; }
  size_t capacity() const { return cap_; }
  size_t peak() const { return peak_; }
  size_t used() const { return used_; }

 private:
  void* base_ = nullptr;
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

enum ReqState { PENDING = 0, RESIDENT = 1, DONE = 2, FAILED = 3, CANCELLED = 4 };

struct Req {
  uint64_t id = 0;
  kpm_handle h = nullptr;
  kpm_params p{};
  int K = 0;
  bool fp32 = false, cplx = false, solo = false;
  int Rp = 0, G = 0, steps = 0, step = 0;
  ReqState state = PENDING;
  bool cancel = false;
  kpm_status status = KPM_OK;
  std::string error;
  size_t off = 0, bytes = 0;
  // device buffers inside the arena
  void* v[2] = {nullptr, nullptr};
  double *sums = nullptr, *per_vec = nullptr, *mu = nullptr, *E = nullptr, *rho = nullptr,
         *dos_work = nullptr, *ring = nullptr;
  RunParams* prm = nullptr;
  ScalarBlock* sc = nullptr;
  void *hs = nullptr, *ds = nullptr;
  RunParams host_prm{};
  StepArgs args{};
  int block = 0, grid = 0, ring_slots = 0;
  cudaStream_t st = nullptr;  // the stream this request runs on
  double a = 1.0, b = 0.0;
  std::vector<double> out_mu, out_E, out_rho;
  double t_submit = 0, t_admit = 0, t_done = 0;
  // large requests: completion of the chunk in flight (ending at step inflight_end)
  cudaEvent_t ev = nullptr;
  bool inflight = false;
  int inflight_end = 0;
  ~Req() {
    if (ev) cudaEventDestroy(ev);
  }
};

uint64_t group_key(const Req* r) {
  const kpm_handle_s* h = r->h;
  uint64_t k = (uint64_t)r->fp32 | ((uint64_t)r->cplx << 1) | ((uint64_t)h->stencil << 2) |
               ((uint64_t)h->geom.dims << 3) | ((uint64_t)h->has_hop << 5) |
               ((uint64_t)h->has_onsite << 6) | ((uint64_t)h->ell_w << 7) |
               ((uint64_t)r->Rp << 12);
  return k;
}

}  // namespace

struct kpm_server_s {
  int device = 0;
  int steps_per_tick = 32;
  int C = 4;
  Arena arena;
  cudaStream_t stream = nullptr;                // batched groups
  cudaStream_t solo_streams[SOLO_STREAMS] = {};  // large requests (round robin)
  cudaEvent_t ev_setup = nullptr;                // set-up of a tick's admitted requests
  BatchTask* d_tasks = nullptr;
  BatchTask* h_tasks = nullptr;  // pinned staging
  int* d_queue = nullptr;
  int max_tasks = 4096;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::vector<Req*> resident;
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  // statistics
  uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, ticks = 0;
  std::vector<double> latencies;
  double t_first = 0, t_last = 0;
  int peak_resident = 0;
};

namespace {

size_t layout(Req* r, bool assign, char* base) {
  const kpm_handle_s* h = r->h;
  const size_t esz = elem_bytes(r->fp32, r->cplx);
  const int M = r->p.M, R = r->p.R;
  size_t hs_b = 0, ds_b = 0;
  scaled_operator_bytes(h, r->fp32, &hs_b, &ds_b);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = al(o + std::max<size_t>(bytes, 1));
    return at;
  };
  const size_t o_v0 = take((size_t)h->n * r->Rp * esz);
  const size_t o_v1 = take((size_t)h->n * r->Rp * esz);
  const size_t o_sums = take((size_t)r->steps * 2 * r->Rp * 8);
  const size_t o_pv = take((size_t)R * M * 8);
  const size_t o_mu = take((size_t)M * 8);
  const size_t o_E = take((size_t)std::max(r->K, 1) * 8);
  const size_t o_rho = take((size_t)std::max(r->K, 1) * 8);
  const size_t o_dw = take(((size_t)M + 4 * (size_t)std::max(r->K, 1)) * 8);
  const size_t o_prm = take(sizeof(RunParams));
  const size_t o_sc = take(sizeof(ScalarBlock));
  const size_t o_hs = take(hs_b);
  const size_t o_ds = take(ds_b);
  const size_t o_ring = take(r->solo ? (size_t)r->ring_slots * r->grid * 2 * r->Rp * 8 : 0);
  if (assign) {
    char* p = base + r->off;
    r->v[0] = p + o_v0;
    r->v[1] = p + o_v1;
    r->sums = (double*)(p + o_sums);
    r->per_vec = (double*)(p + o_pv);
    r->mu = (double*)(p + o_mu);
    r->E = (double*)(p + o_E);
    r->rho = (double*)(p + o_rho);
    r->dos_work = (double*)(p + o_dw);
    r->prm = (RunParams*)(p + o_prm);
    r->sc = (ScalarBlock*)(p + o_sc);
    r->hs = p + o_hs;
    r->ds = p + o_ds;
    r->ring = r->solo ? (double*)(p + o_ring) : nullptr;
  }
  return o;
}

// Operator arguments and traversal; for solo requests also the full-GPU grid.
void prepare(kpm_server_s* s, Req* r) {
  operator_args(r->args, r->h, r->hs, r->ds, r->sc, r->Rp, r->G);
  if (r->solo) {
    plan_step_grid(r->h, r->fp32, r->args, &r->block, &r->grid);
  } else {
    // the batched kernel splits the rows among the cluster's CTAs
    const kpm_handle_s* h = r->h;
    StepArgs& a = r->args;
    const int spi = 256 / a.Gt;
    a.line_len = 0;
    a.lines = 0;
    a.line_L1 = h->geom.L[1];
    a.passes = (h->n + spi - 1) / spi;
    if (h->stencil && h->geom.dims >= 2 && h->geom.L[0] >= 4) {
      const int64_t lines = h->n / h->geom.L[0];
      const int64_t padded = (lines + spi - 1) / spi * spi;
      if (lines >= spi && 8 * (padded - lines) <= lines) {
        a.line_len = h->geom.L[0];
        a.lines = (int)lines;
        a.passes = padded / spi * (int64_t)h->geom.L[0];
      }
    }
    a.chunk = 2;
  }
  (void)s;
}

cudaError_t solo_advance(kpm_server_s* s, Req* r, int b, int e) {
  cudaStream_t st = r->st;
  (void)s;
  cudaError_t err = cudaSuccess;
  StepArgs a = r->args;
  const LaunchCfg cfg{r->block, r->grid};
  for (int step = b; step < e && err == cudaSuccess; ++step) {
    if (step == 0) err = launch_rng_init(r->fp32, r->cplx, a.n, r->Rp, r->prm, r->v[0], st);
    if (err != cudaSuccess) break;
    a.x = r->v[step & 1];
    a.y = r->v[(step + 1) & 1];
    a.w = a.y;
    a.partial = r->ring + (size_t)(step % r->ring_slots) * r->grid * 2 * r->Rp;
    a.reverse = (step & 1) ^ 1;  // alternate sweep directions (see StepArgs)
    const StepMode mode = step == 0 ? MODE_FIRST : MODE_STEP;
    err = r->fp32 ? launch_step_f32(r->h->stencil, r->cplx, mode, a, cfg, st)
                  : launch_step_f64(r->h->stencil, r->cplx, mode, a, cfg, st);
  }
  if (err == cudaSuccess)
    err = launch_reduce_ring(r->ring, r->ring_slots, b, e - b, r->grid, r->Rp, r->prm, r->steps,
                             r->sums, st);
  if (err == cudaSuccess && e == r->steps)
    err = launch_finalize(r->sums, 1, r->steps, r->p.R, r->Rp, a.n, r->p.M, r->per_vec, r->mu,
                          r->prm, st);
  return err;
}

void fail_req(Req* r, kpm_status st, const std::string& msg) {
  r->status = st;
  r->error = msg;
  r->state = FAILED;
}

void worker_loop(kpm_server_s* s) {
  cudaSetDevice(s->device);
  std::vector<Req*> admitted;
  for (;;) {
    admitted.clear();
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return s->stop || !s->pending.empty() || !s->resident.empty(); });
      if (s->stop) break;
      // admission, first come first served, bounded by the arena (HBM budget)
      while (!s->pending.empty()) {
        Req* r = s->pending.front();
        if (r->cancel) {
          s->pending.pop_front();
          r->state = CANCELLED;
          ++s->cancelled;
          s->cv_done.notify_all();
          continue;
        }
        if ((int)s->resident.size() >= s->max_tasks) break;
        size_t off = 0;
        if (!s->arena.alloc(r->bytes, &off)) break;
        s->pending.pop_front();
        r->off = off;
        r->state = RESIDENT;
        r->t_admit = now_s();
        layout(r, true, s->arena.base());
        s->resident.push_back(r);
        admitted.push_back(r);
      }
      s->peak_resident = std::max(s->peak_resident, (int)s->resident.size());
    }
    cudaStream_t st = s->stream;
    // set-up of the newly admitted: parameters and the scaled operator
    for (Req* r : admitted) {
      r->host_prm = RunParams{};
      r->host_prm.a = r->a;
      r->host_prm.b = r->b;
      r->host_prm.seed = (unsigned long long)r->p.seed;
      r->host_prm.R = r->p.R;
      r->host_prm.S = 1;
      r->host_prm.M = r->p.M;
      cudaError_t e = cudaMemcpyAsync(r->prm, &r->host_prm, sizeof(RunParams),
                                      cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = prescale_into(r->h, r->fp32, r->prm, r->hs, r->ds, r->sc, st);
      if (e == cudaSuccess) prepare(s, r);
      if (e != cudaSuccess) fail_req(r, KPM_ECUDA, cudaGetErrorString(e));
    }
    // the large requests' streams wait for the set-up done on the main stream
    bool any_solo = false;
    for (Req* r : admitted) any_solo |= r->solo;
    if (any_solo) cudaEventRecord(s->ev_setup, st);
    for (Req* r : admitted) {
      r->st = r->solo ? s->solo_streams[r->id % SOLO_STREAMS] : st;
      if (r->solo) {
        cudaError_t e = r->ev ? cudaSuccess : cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(r->st, s->ev_setup, 0);
        if (e != cudaSuccess) fail_req(r, KPM_ECUDA, cudaGetErrorString(e));
      }
    }
    // advance: batched groups, then the large requests
    std::vector<Req*> live;
    for (Req* r : s->resident)
      if (r->state == RESIDENT && !r->cancel) live.push_back(r);
    std::map<uint64_t, std::vector<Req*>> groups;
    for (Req* r : live)
      if (!r->solo) groups[group_key(r)].push_back(r);
    int ntask = 0, gi = 0;
    cudaError_t err = cudaSuccess;
    std::vector<std::pair<int, int>> spans;  // per group: first task, count
    for (auto& kv : groups) {
      auto& rs = kv.second;
      std::stable_sort(rs.begin(), rs.end(), [](const Req* x, const Req* y) {
        return (double)x->h->n * (x->steps - x->step) > (double)y->h->n * (y->steps - y->step);
      });
      spans.emplace_back(ntask, (int)rs.size());
      for (Req* r : rs) {
        BatchTask& t = s->h_tasks[ntask++];
        memset(&t, 0, sizeof(t));
        t.a = r->args;
        t.v[0] = r->v[0];
        t.v[1] = r->v[1];
        t.sums = r->sums;
        t.per_vec = r->per_vec;
        t.mu = r->mu;
        t.step_begin = r->step;
        t.step_end = std::min(r->step + s->steps_per_tick, r->steps);
        t.M = r->p.M;
        t.R = r->p.R;
        t.seed = (unsigned long long)r->p.seed;
      }
    }
    if (ntask > 0)
      err = cudaMemcpyAsync(s->d_tasks, s->h_tasks, ntask * sizeof(BatchTask),
                            cudaMemcpyHostToDevice, st);
    if (groups.size() > (size_t)MAX_GROUPS) err = cudaErrorInvalidValue;
    if (err == cudaSuccess && !groups.empty())
      err = cudaMemsetAsync(s->d_queue, 0, groups.size() * sizeof(int), st);
    for (auto& kv : groups) {
      if (err != cudaSuccess) break;
      const auto span = spans[gi];
      const Req* r0 = kv.second.front();
      const StepArgs& proto = s->h_tasks[span.first].a;
      const int nclu = r0->fp32 ? max_clusters_batch_f32(r0->cplx, proto, s->C)
                                : max_clusters_batch_f64(r0->cplx, proto, s->C);
      const int grid = std::max(1, std::min(span.second, std::max(nclu, 1))) * s->C;
      err = r0->fp32 ? launch_batch_f32(r0->cplx, proto, s->d_tasks + span.first, span.second,
                                        s->d_queue + gi, grid, s->C, st)
                     : launch_batch_f64(r0->cplx, proto, s->d_tasks + span.first, span.second,
                                        s->d_queue + gi, grid, s->C, st);
      ++gi;
    }
    bool progressed = !groups.empty();
    std::vector<std::pair<Req*, int>> advanced;  // batched requests, and large requests enqueued now
    std::vector<Req*> enqueued;
    for (Req* r : live) {
      if (!r->solo) {
        advanced.emplace_back(r, std::min(r->step + s->steps_per_tick, r->steps));
        continue;
      }
      if (r->inflight || err != cudaSuccess) continue;
      const int e = std::min(r->step + s->steps_per_tick * SOLO_CHUNK_TICKS, r->steps);
      cudaError_t se = solo_advance(s, r, r->step, e);
      if (se != cudaSuccess) {
        cudaStreamSynchronize(r->st);  // nothing of it may still run when its memory is freed
        cudaGetLastError();
        fail_req(r, KPM_ECUDA, cudaGetErrorString(se));
        continue;
      }
      r->inflight_end = e;
      enqueued.push_back(r);
      progressed = true;
    }
    // DOS and result copies of the requests that finish with this tick's work,
    // each on the stream that advanced it
    std::vector<std::pair<Req*, int>> finishing = advanced;
    for (Req* r : enqueued) finishing.emplace_back(r, r->inflight_end);
    for (auto& pe : finishing) {
      Req* r = pe.first;
      if (pe.second != r->steps || (!r->solo && err != cudaSuccess)) continue;
      cudaStream_t rs = r->st;
      cudaError_t fe = cudaSuccess;
      if (r->K > 0)
        fe = launch_dos(r->mu, r->p.M, r->a, r->b, r->K, KPM_KERNEL_JACKSON, 0.0, r->E, r->rho,
                        r->dos_work, rs);
      r->out_mu.resize(r->p.M);
      if (fe == cudaSuccess)
        fe = cudaMemcpyAsync(r->out_mu.data(), r->mu, r->p.M * sizeof(double),
                             cudaMemcpyDeviceToHost, rs);
      if (fe == cudaSuccess && r->K > 0) {
        r->out_E.resize(r->K);
        r->out_rho.resize(r->K);
        fe = cudaMemcpyAsync(r->out_E.data(), r->E, r->K * sizeof(double), cudaMemcpyDeviceToHost, rs);
        if (fe == cudaSuccess)
          fe = cudaMemcpyAsync(r->out_rho.data(), r->rho, r->K * sizeof(double),
                               cudaMemcpyDeviceToHost, rs);
      }
      if (fe != cudaSuccess) {
        if (r->solo)
          fail_req(r, KPM_ECUDA, cudaGetErrorString(fe));  // still waits for its chunk in flight
        else
          err = fe;
      }
    }
    for (Req* r : enqueued) {
      cudaError_t e = cudaEventRecord(r->ev, r->st);
      if (e != cudaSuccess) {
        fail_req(r, KPM_ECUDA, cudaGetErrorString(e));
        cudaStreamSynchronize(r->st);  // nothing of it may still run when its memory is freed
        continue;
      }
      r->inflight = true;
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    const double t = now_s();
    {
      std::lock_guard<std::mutex> lock(s->mu);
      ++s->ticks;
      // large requests whose chunk in flight has completed
      for (Req* r : s->resident) {
        if (!r->solo || !r->inflight) continue;
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) continue;
        r->inflight = false;
        progressed = true;
        if (r->state == FAILED) continue;
        if (q != cudaSuccess) {
          cudaGetLastError();
          fail_req(r, KPM_ECUDA, cudaGetErrorString(q));
          continue;
        }
        r->step = r->inflight_end;
        if (r->step == r->steps) {
          bool bad = false;
          for (double m : r->out_mu) bad |= !(fabs(m) <= 1.0 + 1e-6);
          r->status = bad ? KPM_EDIVERGE : KPM_OK;
          if (bad) r->error = "a moment left [-1, 1]: the bounds do not enclose the spectrum";
          r->state = DONE;
          r->t_done = now_s();
        }
      }
      for (auto& pe : advanced) {
        Req* r = pe.first;
        if (err != cudaSuccess) {
          fail_req(r, KPM_ECUDA, cudaGetErrorString(err));
          continue;
        }
        r->step = pe.second;
        if (r->step == r->steps) {
          bool bad = false;
          for (double m : r->out_mu) bad |= !(fabs(m) <= 1.0 + 1e-6);
          r->status = bad ? KPM_EDIVERGE : KPM_OK;
          if (bad) r->error = "a moment left [-1, 1]: the bounds do not enclose the spectrum";
          r->state = DONE;
          r->t_done = t;
        }
      }
      // retire finished, failed and cancelled requests
      std::vector<Req*> keep;
      for (Req* r : s->resident) {
        if (r->state == RESIDENT && r->cancel && !r->inflight) {
          r->state = CANCELLED;
          ++s->cancelled;
        }
        if (r->state == RESIDENT || r->inflight) {
          keep.push_back(r);
          continue;
        }
        s->arena.release(r->off, r->bytes);
        if (r->state == DONE) {
          ++s->completed;
          s->latencies.push_back(r->t_done - r->t_submit);
          s->t_last = std::max(s->t_last, r->t_done);
        } else if (r->state == FAILED) {
          ++s->failed;
        }
      }
      s->resident.swap(keep);
      s->cv_done.notify_all();
    }
    if (err != cudaSuccess) cudaGetLastError();
    // only large requests in flight and nothing to do: poll again shortly
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

}  // namespace

extern "C" {

kpm_status kpm_server_create(size_t hbm_budget_bytes, int steps_per_tick, int cluster,
                             kpm_server* out) {
  if (!out) return fail(KPM_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20)) return fail(KPM_EINVAL, "budget below 1 MiB");
  if (steps_per_tick < 1 || steps_per_tick > 64) return fail(KPM_EINVAL, "steps_per_tick in 1..64");
  if (cluster < 1 || cluster > 16 || (cluster & (cluster - 1)))
    return fail(KPM_EINVAL, "cluster must be a power of two <= 16");
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(KPM_ECUDA, "no usable CUDA device");
  }
  auto* s = new kpm_server_s();
  KPM_CUDA(cudaGetDevice(&s->device));
  s->steps_per_tick = steps_per_tick;
  s->C = cluster;
  cudaError_t e = s->arena.init(hbm_budget_bytes);
  // the batched groups (many small requests) get the highest stream priority,
  // the large requests the lowest: the block scheduler then starts the small
  // requests' CTAs first and fills the rest of the GPU with the large ones
  int prio_low = 0, prio_high = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_setup, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_tasks, s->max_tasks * sizeof(BatchTask));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_tasks, s->max_tasks * sizeof(BatchTask));
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_queue, MAX_GROUPS * sizeof(int));
  for (int k = 0; k < SOLO_STREAMS && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithPriority(&s->solo_streams[k], cudaStreamNonBlocking, prio_low);
  if (e != cudaSuccess) {
    kpm_status st = cuda_fail(e, "server set-up");
    s->arena.destroy();
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->d_tasks) cudaFree(s->d_tasks);
    if (s->h_tasks) cudaFreeHost(s->h_tasks);
    if (s->d_queue) cudaFree(s->d_queue);
    delete s;
    return st;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return KPM_OK;
}

kpm_status kpm_server_submit(kpm_server s, kpm_handle h, const kpm_params* p, int K,
                             uint64_t* req_id) {
  if (!s || !h || !p || !req_id) return fail(KPM_EINVAL, "NULL argument");
  if (p->M < 2 || (p->M & 1)) return fail(KPM_EINVAL, "M must be even and >= 2");
  if (p->R < 1) return fail(KPM_EINVAL, "R must be >= 1");
  if (p->S > 1 || p->user_v0 || p->s0 != 0)
    return fail(KPM_EINVAL, "served requests take S = 1, s0 = 0 and no user_v0");
  if (p->precision != KPM_FP64 && p->precision != KPM_FP32_VEC_FP64_MOM)
    return fail(KPM_EINVAL, "bad precision");
  if (!(p->a > 0.0) || !isfinite(p->a) || !isfinite(p->b)) return fail(KPM_EINVAL, "bad a or b");
  if (K < 0 || K > (1 << 20)) return fail(KPM_EINVAL, "bad K");
  if (h->device != s->device) return fail(KPM_EINVAL, "handle on another device");
  if (h->dense) return fail(KPM_EINVAL, "dense handles are not served (use kpm_moments)");
  auto* r = new Req();
  r->h = h;
  r->p = *p;
  r->K = K;
  r->a = p->a;
  r->b = p->b;
  r->fp32 = p->precision == KPM_FP32_VEC_FP64_MOM;
  r->cplx = h->cplx;
  padded_width(p->R, r->fp32, r->cplx, &r->Rp, &r->G);
  r->steps = p->M / 2;
  r->solo = 3 * (size_t)h->n * r->Rp * elem_bytes(r->fp32, r->cplx) >= SOLO_STEP_BYTES ||
            r->G > 256;
  if (r->solo) {
    // grid of the full-GPU fused step for this shape (sets the ring size)
    StepArgs probe{};
    operator_args(probe, h, nullptr, nullptr, nullptr, r->Rp, r->G);
    plan_step_grid(h, r->fp32, probe, &r->block, &r->grid);
    r->ring_slots = s->steps_per_tick * SOLO_CHUNK_TICKS;
  }
  r->bytes = layout(r, false, nullptr);
  if (r->bytes > s->arena.capacity()) {
    delete r;
    return fail(KPM_ENOMEM, "request larger than the server's HBM budget");
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    ++s->submitted;
    if (s->t_first == 0) s->t_first = r->t_submit;
    *req_id = r->id;
  }
  s->cv_work.notify_one();
  return KPM_OK;
}

kpm_status kpm_server_wait(kpm_server s, uint64_t id, double timeout_s) {
  if (!s) return fail(KPM_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(KPM_EINVAL, "unknown request id");
  Req* r = it->second;
  auto ready = [&] { return r->state == DONE || r->state == FAILED || r->state == CANCELLED; };
  if (timeout_s < 0) {
    s->cv_done.wait(lock, ready);
  } else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready)) {
    return fail(KPM_ETIMEOUT, "request not finished within the timeout");
  }
  return KPM_OK;
}

kpm_status kpm_server_poll(kpm_server s, uint64_t id, double* mu, double* E, double* rho,
                           double* latency_s) {
  if (!s) return fail(KPM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(KPM_EINVAL, "unknown request id");
  Req* r = it->second;
  if (r->state == PENDING || r->state == RESIDENT) return fail(KPM_ENOTREADY, "request in flight");
  kpm_status st = r->status;
  if (r->state == CANCELLED) st = fail(KPM_EINVAL, "request was cancelled");
  if (r->state == FAILED) st = fail(r->status, r->error);
  if (r->state == DONE) {
    if (mu) memcpy(mu, r->out_mu.data(), r->out_mu.size() * sizeof(double));
    if (E && !r->out_E.empty()) memcpy(E, r->out_E.data(), r->out_E.size() * sizeof(double));
    if (rho && !r->out_rho.empty()) memcpy(rho, r->out_rho.data(), r->out_rho.size() * sizeof(double));
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    if (st != KPM_OK) set_error(r->error);
  }
  s->reqs.erase(it);
  delete r;
  return st;
}

kpm_status kpm_server_cancel(kpm_server s, uint64_t id) {
  if (!s) return fail(KPM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(KPM_EINVAL, "unknown request id");
  it->second->cancel = true;
  s->cv_work.notify_one();
  return KPM_OK;
}

kpm_status kpm_server_stats(kpm_server s, kpm_server_stats_t* out) {
  if (!s || !out) return fail(KPM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->cancelled = s->cancelled;
  out->ticks = s->ticks;
  out->peak_resident = s->peak_resident;
  out->peak_bytes = s->arena.peak();
  out->budget_bytes = s->arena.capacity();
  if (!s->latencies.empty()) {
    std::vector<double> l = s->latencies;
    std::sort(l.begin(), l.end());
    auto q = [&](double f) {
      const double pos = f * (l.size() - 1);
      const size_t i = (size_t)pos;
      const double w = pos - i;
      return i + 1 < l.size() ? l[i] * (1 - w) + l[i + 1] * w : l[i];
    };
    out->p50_s = q(0.50);
    out->p99_s = q(0.99);
    out->max_s = l.back();
    double sum = 0;
    for (double x : l) sum += x;
    out->mean_s = sum / l.size();
    const double span = s->t_last - s->t_first;
    out->solves_per_s = span > 0 ? s->completed / span : 0.0;
  }
  return KPM_OK;
}

void kpm_server_destroy(kpm_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (int k = 0; k < SOLO_STREAMS; ++k) cudaStreamSynchronize(s->solo_streams[k]);
  for (auto& kv : s->reqs) delete kv.second;
  s->arena.destroy();
  cudaStreamDestroy(s->stream);
  for (int k = 0; k < SOLO_STREAMS; ++k) cudaStreamDestroy(s->solo_streams[k]);
  if (s->ev_setup) cudaEventDestroy(s->ev_setup);
  cudaFree(s->d_tasks);
  cudaFreeHost(s->h_tasks);
  cudaFree(s->d_queue);
  delete s;
}

}  // extern "C"
