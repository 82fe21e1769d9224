// C ABI of the batched persistent launch (kpm_batch_*): many independent KPM
// solves of uneven size advanced by one cluster kernel launch that is captured
// once into a CUDA graph and replayed, with an autotuner choosing the cluster
// size, the number of resident clusters, the traversal chunk and the R-tiling
// (an instance's vector columns split into independent tasks).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "kpm_batch.cuh"

using namespace kpm;

namespace {
constexpr int FORM_GLOBAL = 0, FORM_RESIDENT = 1, FORM_STAGED = 2;
}

struct BatchConfig {
  int C = 4;          // CTAs per cluster
  int chunk = 4;      // passes per traversal chunk
  int frac = 100;     // percent of the co-resident clusters launched
  int rtiles = 1;     // column tiles of a tiled instance (divides the chunks per row)
  int top = 0;        // the `top` instances of largest work are tiled (<= 0: all)
  int res = 0;        // vector rows: 0 global memory, 1 resident in the clusters' shared
                      // memory, 2 staged through shared-memory rings (chunk: tile size)
  int tpr = 1;        // threads per row relative to the 32-byte chunk (2: 16-byte chunks)
};

constexpr int MAX_RTILES = 4;

struct kpm_batch_s {
  int device = 0;
  int count = 0;
  bool fp32 = false, cplx = false;
  int R = 0, Rp = 0, G = 0;
  std::vector<kpm_handle> handles;   // not owned
  std::vector<int> M;                // per instance (original order)
  std::vector<size_t> mu_off;        // offsets of each instance's moments in the output
  size_t mu_total = 0;
  std::vector<int> order;            // instance slots in decreasing work
  std::vector<BatchTask> inst_tasks; // one untiled task per instance (instance order)
  std::vector<BatchTask> host_tasks; // task slot order of the current configuration
  BatchTask* d_tasks = nullptr;
  int* d_queue = nullptr;            // [0] task queue, [1 + i] tiles finished of instance i
  void* d_pool = nullptr;            // vectors, sums, per-vector moments, operators
  double* d_mu = nullptr;            // [mu_total] in instance order (inside the pool)
  StepArgs proto{};                  // template-selecting prototype (first instance)
  BatchConfig cfg;
  int grid = 0;
  bool tuned = false;
  cudaGraphExec_t exec = nullptr;
  BatchConfig exec_cfg;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double last_ms = 0.0;
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int vec_cols(bool fp32, bool cplx) { return fp32 ? (cplx ? 4 : 8) : (cplx ? 1 : 2); }

std::string device_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  return p.name;
}

// Traversal of one instance split among C CTAs (same rules as the single fused step).
void plan_instance(StepArgs& a, const kpm_handle_s* h, int chunk) {
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
  a.chunk = chunk;
}

// Whether 16-byte chunks (twice the threads per row) apply: real FP32 stencils.
bool half_chunks_ok(const kpm_batch_s* b) {
  return b->fp32 && !b->cplx && b->handles[0]->stencil;
}

// Launch prototype of configuration c: chunks per row and per task.
StepArgs cfg_proto(const kpm_batch_s* b, const BatchConfig& c) {
  StepArgs a = b->inst_tasks[b->order[0]].a;
  a.G = b->G * c.tpr;
  a.Gt = a.G / std::max(1, c.rtiles);
  return a;
}

int max_clusters(kpm_batch_s* b, const BatchConfig& c) {
  const StepArgs a = cfg_proto(b, c);
  if (c.tpr == 2) return max_clusters_batch_f32h(a, c.C);
  return b->fp32 ? max_clusters_batch_f32(b->cplx, a, c.C)
                 : max_clusters_batch_f64(b->cplx, a, c.C);
}

// Rows per CTA the resident form needs at cluster size C (the largest instance).
int64_t res_rows_cap(const kpm_batch_s* b, int C) {
  int64_t cap = 1;
  for (const kpm_handle_s* h : b->handles) cap = std::max<int64_t>(cap, (h->n + C - 1) / C);
  return cap;
}

// Co-resident clusters of the resident form at cluster size C (0: the
// operator is not a stencil or the largest instance does not fit).
int max_clusters_res(kpm_batch_s* b, int C) {
  const StepArgs& a = b->inst_tasks[b->order[0]].a;
  const int64_t cap = res_rows_cap(b, C);
  return b->fp32 ? max_clusters_batch_res_f32(b->cplx, a, C, cap)
                 : max_clusters_batch_res_f64(b->cplx, a, C, cap);
}

// Tile shape of the staged form: tiles of 2^Tl rows of about 4 KB x `chunk`
// (at least one pass of the 256 threads), 2^Sl stages of v_n (about 64 KB)
// and 2^SWl of v_{n-1} (about 32 KB), so that two CTAs fit an SM.
struct StgShape {
  int Tl, Sl, SWl;
};
StgShape stg_shape(const kpm_batch_s* b, int chunk) {
  const int rowB = b->G * (b->fp32 ? 32 : 16);
  int Tl = 0;
  while ((1 << Tl) < 256 / b->G || (1 << Tl) * rowB < 4096 * std::max(1, chunk)) ++Tl;
  const size_t tileB = (size_t)rowB << Tl;
  int Sl = 3, SWl = 3;
  while (Sl > 2 && ((size_t)1 << Sl) * tileB > 64 * 1024) --Sl;
  while (SWl > 1 && ((size_t)1 << SWl) * tileB > 32 * 1024) --SWl;
  // KPM_BATCH_STG="Sl,SWl" sets the ring depths (log2 stages, 2..4 and 1..4)
  if (const char* env = getenv("KPM_BATCH_STG")) {
    int a = 0, c = 0;
    if (sscanf(env, "%d,%d", &a, &c) == 2 && a >= 2 && a <= 4 && c >= 1 && c <= 4) {
      Sl = a;
      SWl = c;
    }
  }
  return {Tl, Sl, SWl};
}

// Whether the staged form applies: stencil operators, rows of at most 32 chunks.
bool staged_ok(const kpm_batch_s* b) { return b->handles[0]->stencil && b->G <= 32; }

int max_clusters_stg(kpm_batch_s* b, const BatchConfig& c) {
  if (!staged_ok(b)) return 0;
  const StgShape sh = stg_shape(b, c.chunk);
  const StepArgs& a = b->inst_tasks[b->order[0]].a;
  return b->fp32 ? max_clusters_batch_stg_f32(b->cplx, a, c.C, sh.Tl, sh.Sl, sh.SWl)
                 : max_clusters_batch_stg_f64(b->cplx, a, c.C, sh.Tl, sh.Sl, sh.SWl);
}

int cfg_clusters(kpm_batch_s* b, const BatchConfig& c) {
  if (c.res == FORM_STAGED) return max_clusters_stg(b, c);
  return c.res ? max_clusters_res(b, c.C) : max_clusters(b, c);
}

kpm_status build_graph(kpm_batch_s* b, const BatchConfig& c) {
  if (b->exec && b->exec_cfg.C == c.C && b->exec_cfg.chunk == c.chunk &&
      b->exec_cfg.frac == c.frac && b->exec_cfg.rtiles == c.rtiles && b->exec_cfg.top == c.top &&
      b->exec_cfg.res == c.res && b->exec_cfg.tpr == c.tpr)
    return KPM_OK;
  if (c.tpr != 1 && (c.tpr != 2 || !half_chunks_ok(b) || c.res))
    return fail(KPM_EINVAL,
                "twice the threads per row needs a real FP32 stencil batch in the global-memory form");
  const int Geff = b->G * c.tpr;
  if (c.rtiles < 1 || c.rtiles > MAX_RTILES || Geff % c.rtiles)
    return fail(KPM_EINVAL, "R-tiles must divide the chunks per row");
  if (c.res && c.rtiles > 1)
    return fail(KPM_EINVAL, "the resident form runs untiled instances (R-tiles 1)");
  if (c.res && !b->handles[0]->stencil)
    return fail(KPM_EINVAL, "the resident and staged forms take stencil operators only");
  if (c.res == FORM_STAGED && !staged_ok(b))
    return fail(KPM_EINVAL, "the staged form takes rows of at most 32 chunks");
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  // tasks of this configuration: instances in decreasing work, the `top`
  // largest split into rtiles column tiles (consecutive in the queue)
  b->host_tasks.clear();
  const int ntiled = c.rtiles > 1 ? (c.top <= 0 ? b->count : std::min(c.top, b->count)) : 0;
  for (int k = 0; k < b->count; ++k) {
    const int i = b->order[k];
    const int T = k < ntiled ? c.rtiles : 1;
    for (int j = 0; j < T; ++j) {
      BatchTask t = b->inst_tasks[i];
      t.a.G = Geff;
      t.a.Gt = Geff / T;
      plan_instance(t.a, b->handles[i], c.chunk);
      t.ycol = j;
      t.ntiles = T;
      t.tiles_done = b->d_queue + 1 + i;
      b->host_tasks.push_back(t);
    }
  }
  // the kernel's shared memory is sized for the widest task
  b->proto = b->host_tasks.back().a;
  const int ntasks = (int)b->host_tasks.size();
  const int nclu = cfg_clusters(b, c);
  if (nclu <= 0)
    return fail(KPM_EINVAL, "cluster size " + std::to_string(c.C) + " cannot be launched" +
                                (c.res ? " with the vectors resident in shared memory" : ""));
  const int use = std::max(1, std::min(ntasks, nclu * c.frac / 100));
  b->grid = use * c.C;
  KPM_CUDA(cudaMemcpy(b->d_tasks, b->host_tasks.data(), b->host_tasks.size() * sizeof(BatchTask),
                      cudaMemcpyHostToDevice));
  const uint64_t before = g_launches.load();
  KPM_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(b->d_queue, 0, (1 + (size_t)b->count) * sizeof(int), b->cap_stream);
  if (e == cudaSuccess)
    e = cudaEventRecordWithFlags(b->ev[0], b->cap_stream, cudaEventRecordExternal);
  if (e == cudaSuccess && c.res == FORM_STAGED) {
    const StgShape sh = stg_shape(b, c.chunk);
    e = b->fp32 ? launch_batch_stg_f32(b->cplx, b->proto, b->d_tasks, ntasks, b->d_queue, b->grid,
                                       c.C, sh.Tl, sh.Sl, sh.SWl, b->cap_stream)
                : launch_batch_stg_f64(b->cplx, b->proto, b->d_tasks, ntasks, b->d_queue, b->grid,
                                       c.C, sh.Tl, sh.Sl, sh.SWl, b->cap_stream);
  } else if (e == cudaSuccess && c.res) {
    const int64_t cap = res_rows_cap(b, c.C);
    e = b->fp32 ? launch_batch_res_f32(b->cplx, b->proto, b->d_tasks, ntasks, b->d_queue, b->grid,
                                       c.C, cap, b->cap_stream)
                : launch_batch_res_f64(b->cplx, b->proto, b->d_tasks, ntasks, b->d_queue, b->grid,
                                       c.C, cap, b->cap_stream);
  } else if (e == cudaSuccess && c.tpr == 2) {
    e = launch_batch_f32h(b->proto, b->d_tasks, ntasks, b->d_queue, b->grid, c.C, b->cap_stream);
  } else if (e == cudaSuccess) {
    e = b->fp32 ? launch_batch_f32(b->cplx, b->proto, b->d_tasks, ntasks, b->d_queue, b->grid,
                                   c.C, b->cap_stream)
                : launch_batch_f64(b->cplx, b->proto, b->d_tasks, ntasks, b->d_queue, b->grid,
                                   c.C, b->cap_stream);
  }
  if (e == cudaSuccess)
    e = cudaEventRecordWithFlags(b->ev[1], b->cap_stream, cudaEventRecordExternal);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  g_launches.fetch_sub(g_launches.load() - before);  // captured, not yet run
  if (e != cudaSuccess) {
    b->exec = nullptr;
    cudaGetLastError();
    return cuda_fail(e, "capture of the batch graph");
  }
  b->exec_cfg = c;
  return KPM_OK;
}

kpm_status replay(kpm_batch_s* b, cudaStream_t st) {
  KPM_CUDA(cudaGraphLaunch(b->exec, st));
  g_launches.fetch_add(1);
  return KPM_OK;
}

std::string tune_key(const kpm_batch_s* b) {
  uint64_t rows = 0, work = 0;
  for (int i = 0; i < b->count; ++i) {
    rows += (uint64_t)b->handles[i]->n;
    work += (uint64_t)b->handles[i]->n * (uint64_t)b->M[i];
  }
  const kpm_handle_s* h = b->handles[0];
  char buf[512];
  snprintf(buf, sizeof(buf), "batch|%s|fp32=%d|cplx=%d|stencil=%d|dims=%d|hop=%d|ds=%d|ell=%d|R=%d|n=%d|rows=%llu|work=%llu",
           device_name(b->device).c_str(), (int)b->fp32, (int)b->cplx, (int)h->stencil,
           h->geom.dims, (int)h->has_hop, (int)h->has_onsite, h->ell_w, b->R, b->count,
           (unsigned long long)rows, (unsigned long long)work);
  return buf;
}

std::string cache_path() {
  const char* p = getenv("KPM_TUNE_CACHE");
  if (p && *p) return p;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/kpm_gb300_autotune.txt";
}

bool cache_lookup(const std::string& key, BatchConfig* c) {
  FILE* f = fopen(cache_path().c_str(), "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    std::string s(line);
    const size_t sep = s.rfind(" = ");
    if (sep == std::string::npos || s.substr(0, sep) != key) continue;
    BatchConfig t;
    const int got = sscanf(s.c_str() + sep + 3, "%d %d %d %d %d %d %d", &t.C, &t.chunk, &t.frac,
                           &t.rtiles, &t.top, &t.res, &t.tpr);
    if (got == 3) t.rtiles = 1;  // entries written before R-tiling was tuned
    if (got <= 4) t.top = 0;
    if (got <= 5) t.res = 0;     // entries written before the resident form was tuned
    if (got <= 6) t.tpr = 1;     // entries written before threads per row were tuned
    if (got >= 3) {
      *c = t;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const std::string& key, const BatchConfig& c) {
  const std::string path = cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return;  // an unwritable cache only costs a re-tune
  fprintf(f, "%s = %d %d %d %d %d %d %d\n", key.c_str(), c.C, c.chunk, c.frac, c.rtiles, c.top,
          c.res, c.tpr);
  fclose(f);
}

}  // namespace

extern "C" {

kpm_status kpm_batch_create(int count, const kpm_handle* handles, const kpm_params* params,
                            kpm_batch* out) {
  if (!out) return fail(KPM_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !handles || !params) return fail(KPM_EINVAL, "empty batch");
  const kpm_handle_s* h0 = handles[0];
  if (!h0) return fail(KPM_EINVAL, "NULL handle");
  const int prec = params[0].precision, R = params[0].R;
  if (prec != KPM_FP64 && prec != KPM_FP32_VEC_FP64_MOM) return fail(KPM_EINVAL, "bad precision");
  if (R < 1) return fail(KPM_EINVAL, "R must be >= 1");
  for (int i = 0; i < count; ++i) {
    const kpm_handle_s* h = handles[i];
    const kpm_params& p = params[i];
    if (!h) return fail(KPM_EINVAL, "NULL handle");
    if (h->dense) return fail(KPM_EINVAL, "dense handles are not batched (use kpm_moments)");
    if (h->device != h0->device || h->cplx != h0->cplx || h->stencil != h0->stencil ||
        h->geom.dims != h0->geom.dims || h->has_hop != h0->has_hop ||
        h->has_onsite != h0->has_onsite || h->ell_w != h0->ell_w)
      return fail(KPM_EINVAL, "all handles of a batch must share device, field and operator kind");
    if (p.precision != prec || p.R != R)
      return fail(KPM_EINVAL, "all instances of a batch must share precision and R");
    if (p.M < 2 || (p.M & 1)) return fail(KPM_EINVAL, "M must be even and >= 2");
    if (!(p.a > 0.0) || !isfinite(p.a) || !isfinite(p.b)) return fail(KPM_EINVAL, "bad a or b");
    if (p.user_v0 || (p.S > 1) || p.s0 != 0)
      return fail(KPM_EINVAL, "batched instances take S = 1, s0 = 0 and no user_v0");
  }
  auto* b = new kpm_batch_s();
  b->device = h0->device;
  b->count = count;
  b->fp32 = prec == KPM_FP32_VEC_FP64_MOM;
  b->cplx = h0->cplx;
  b->R = R;
  const int vec = vec_cols(b->fp32, b->cplx);
  int g = (R + vec - 1) / vec, p2 = 1;
  while (p2 < g) p2 <<= 1;
  b->G = p2;
  b->Rp = p2 * vec;
  if (b->G > 256) {
    delete b;
    return fail(KPM_EINVAL, "R too large for the batched kernel");
  }
  b->handles.assign(handles, handles + count);
  auto cleanup = [&](kpm_status s) {
    kpm_batch_destroy(b);
    return s;
  };
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaSetDevice"));

  // pool layout (per instance): v[2], sums, per_vec, RunParams, ScalarBlock, scaled operator
  const size_t esz = (size_t)(b->fp32 ? 4 : 8) * (b->cplx ? 2 : 1);
  const size_t ssz = b->fp32 ? 4 : 8;
  const int c = b->cplx ? 2 : 1;
  std::vector<size_t> off_v(count), off_sums(count), off_pv(count), off_prm(count), off_sc(count),
      off_hs(count), off_ds(count);
  size_t off = 0;
  b->M.resize(count);
  b->mu_off.resize(count);
  for (int i = 0; i < count; ++i) {
    const kpm_handle_s* h = handles[i];
    const int M = params[i].M;
    b->M[i] = M;
    b->mu_off[i] = b->mu_total;
    b->mu_total += M;
    off_v[i] = off;
    off = align_up(off + 2 * (size_t)h->n * b->Rp * esz, 256);
    off_sums[i] = off;
    off = align_up(off + (size_t)(M / 2) * 2 * b->Rp * 8, 256);
    off_pv[i] = off;
    off = align_up(off + (size_t)R * M * 8, 256);
    off_prm[i] = off;
    off = align_up(off + sizeof(RunParams), 256);
    off_sc[i] = off;
    off = align_up(off + sizeof(ScalarBlock), 256);
    off_hs[i] = off;
    size_t hs_bytes = 0, ds_bytes = 0;
    if (h->stencil) {
      if (h->has_hop) hs_bytes = (size_t)h->n * h->geom.dims * c * ssz;
      if (h->has_onsite) ds_bytes = (size_t)h->n * ssz;
    } else {
      hs_bytes = (h->ell_w > 0 ? (size_t)h->n * h->ell_w : (size_t)h->nnz) * c * ssz;
    }
    off = align_up(off + hs_bytes, 256);
    off_ds[i] = off;
    off = align_up(off + ds_bytes, 256);
  }
  const size_t off_mu = off;
  off = align_up(off + b->mu_total * 8, 256);
  e = cudaMalloc(&b->d_pool, std::max<size_t>(off, 256));
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc(batch pool)"));
  e = cudaMalloc((void**)&b->d_tasks, (size_t)count * MAX_RTILES * sizeof(BatchTask));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_queue, (1 + (size_t)count) * sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch set-up"));
  char* pool = (char*)b->d_pool;
  b->d_mu = (double*)(pool + off_mu);

  // scaled operators owned by the batch (independent of later calls on the handles)
  std::vector<BatchTask> tasks(count);
  for (int i = 0; i < count; ++i) {
    kpm_handle_s* h = handles[i];
    const kpm_params& p = params[i];
    RunParams rp{};
    rp.a = p.a;
    rp.b = p.b;
    rp.seed = (unsigned long long)p.seed;
    rp.R = R;
    rp.S = 1;
    rp.M = p.M;
    auto* d_rp = (RunParams*)(pool + off_prm[i]);
    auto* d_sc = (ScalarBlock*)(pool + off_sc[i]);
    e = cudaMemcpy(d_rp, &rp, sizeof(rp), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "copy params"));
    void* hs = pool + off_hs[i];
    void* ds = pool + off_ds[i];
    if (h->stencil)
      e = launch_prescale_stencil(b->fp32, b->cplx, h->n, h->geom.dims, h->d_onsite, h->d_hop,
                                  h->t_re, h->t_im, d_rp, false, h->has_hop ? hs : nullptr,
                                  h->has_onsite ? ds : nullptr, d_sc, nullptr);
    else if (h->ell_w > 0)
      e = launch_prescale_csr(b->fp32, b->cplx, h->n * h->ell_w, h->d_ell_val, d_rp, false, hs,
                              d_sc, nullptr);
    else
      e = launch_prescale_csr(b->fp32, b->cplx, h->nnz, h->d_val, d_rp, false, hs, d_sc, nullptr);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "prescale"));
    BatchTask& t = tasks[i];
    memset(&t, 0, sizeof(t));
    StepArgs& a = t.a;
    a.n = h->n;
    a.Rp = b->Rp;
    a.G = b->G;
    a.Gt = b->G;
    a.sc = d_sc;
    a.geom = h->geom;
    if (h->stencil) {
      a.hs = h->has_hop ? hs : nullptr;
      a.ds = h->has_onsite ? ds : nullptr;
    } else if (h->ell_w > 0) {
      a.col = h->d_ell_col;
      a.vals = hs;
      a.ell_w = h->ell_w;
    } else {
      a.rowptr = h->d_rowptr;
      a.col = h->d_col;
      a.vals = hs;
    }
    plan_instance(a, h, b->cfg.chunk);
    t.v[0] = pool + off_v[i];
    t.v[1] = pool + off_v[i] + (size_t)h->n * b->Rp * esz;
    t.sums = (double*)(pool + off_sums[i]);
    t.per_vec = (double*)(pool + off_pv[i]);
    t.mu = b->d_mu + b->mu_off[i];
    t.step_begin = 0;
    t.step_end = p.M / 2;
    t.M = p.M;
    t.R = R;
    t.seed = (unsigned long long)p.seed;
    t.realisation = 0;
    t.flags = 0;
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "prescale"));
  // longest first: the queue hands instances out in decreasing work
  b->order.resize(count);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    return (double)handles[x]->n * params[x].M > (double)handles[y]->n * params[y].M;
  });
  b->inst_tasks = tasks;
  b->proto = tasks[b->order[0]].a;
  BatchConfig cached;
  if (cache_lookup(tune_key(b), &cached)) {
    b->cfg = cached;
    b->tuned = true;
  }
  *out = b;
  return KPM_OK;
}

kpm_status kpm_batch_run(kpm_batch b, double* mu, void* stream) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  KPM_CUDA(cudaSetDevice(b->device));
  cudaStream_t st = (cudaStream_t)stream;
  kpm_status s = build_graph(b, b->cfg);
  if (s != KPM_OK) return s;
  if ((s = replay(b, st)) != KPM_OK) return s;
  if (!mu) return KPM_OK;
  cudaPointerAttributes at;
  bool dev = false;
  if (cudaPointerGetAttributes(&at, mu) == cudaSuccess)
    dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  else
    cudaGetLastError();
  KPM_CUDA(cudaMemcpyAsync(mu, b->d_mu, b->mu_total * sizeof(double),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (!dev) {
    KPM_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) b->last_ms = ms;
    cudaGetLastError();
    // divergence flags of the instances
    std::vector<BatchTask> back(b->host_tasks.size());
    KPM_CUDA(cudaMemcpy(back.data(), b->d_tasks, back.size() * sizeof(BatchTask),
                        cudaMemcpyDeviceToHost));
    int bad = 0;
    for (auto& t : back) bad |= t.flags;
    if (bad & BATCH_FLAG_TIMEOUT)
      return fail(KPM_ETIMEOUT, "a bounded wait of the staged batch kernel ran out");
    if (bad)
      return fail(KPM_EDIVERGE, "a batched instance left [-1, 1]: its bounds miss the spectrum");
  }
  return KPM_OK;
}

kpm_status kpm_batch_tune(kpm_batch b, int reps, void* stream) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  KPM_CUDA(cudaSetDevice(b->device));
  cudaStream_t st = (cudaStream_t)stream;
  reps = std::max(1, reps);
  const int Cs[] = {1, 2, 4, 8, 16};
  const int chunks[] = {2, 4, 16};
  const int fracs[] = {100, 50};
  BatchConfig best;
  double best_ms = 1e30;
  auto time_cfg = [&](const BatchConfig& c) -> kpm_status {
    if (cfg_clusters(b, c) <= 0) return KPM_OK;
    if (build_graph(b, c) != KPM_OK) {
      cudaGetLastError();
      return KPM_OK;
    }
    if (replay(b, st) != KPM_OK) return fail(KPM_ECUDA, "batch replay failed while tuning");
    double tot = 0.0;
    for (int r = 0; r < reps; ++r) {
      if (replay(b, st) != KPM_OK) return fail(KPM_ECUDA, "batch replay failed while tuning");
      KPM_CUDA(cudaStreamSynchronize(st));
      float ms = 0.f;
      KPM_CUDA(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
      tot += ms;
    }
    const double ms = tot / reps;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
    return KPM_OK;
  };
  // untiled: cluster size, chunk, resident clusters
  for (int C : Cs)
    for (int ch : chunks)
      for (int fr : fracs) {
        BatchConfig c;
        c.C = C;
        c.chunk = ch;
        c.frac = fr;
        kpm_status s_ = time_cfg(c);
        if (s_ != KPM_OK) return s_;
      }
  // twice the threads per row (16-byte chunks; real FP32 stencils): every
  // cluster size and chunk, all co-resident clusters
  if (half_chunks_ok(b))
    for (int C : Cs)
      for (int ch : chunks) {
        BatchConfig c;
        c.C = C;
        c.chunk = ch;
        c.tpr = 2;
        kpm_status s_ = time_cfg(c);
        if (s_ != KPM_OK) return s_;
      }
  // the resident form (stencil operators whose largest instance fits the
  // shared memory of a cluster): every cluster size, all or half of the
  // co-resident clusters (the traversal chunk does not apply)
  if (b->handles[0]->stencil)
    for (int C : Cs)
      for (int fr : fracs) {
        BatchConfig c;
        c.C = C;
        c.frac = fr;
        c.res = 1;
        kpm_status s_ = time_cfg(c);
        if (s_ != KPM_OK) return s_;
      }
  // the staged form (stencil operators): every cluster size, tiles of about
  // 4, 8 and 16 KB
  if (staged_ok(b))
    for (int C : Cs)
      for (int ch : {1, 2, 4}) {
        BatchConfig c;
        c.C = C;
        c.chunk = ch;
        c.res = FORM_STAGED;
        kpm_status s_ = time_cfg(c);
        if (s_ != KPM_OK) return s_;
      }
  // then, if the global-memory form won, R-tiling of the largest instances
  // (all, a half, an eighth, a thirty-second of them) at the best
  // configuration and half its cluster; a tiling is kept only if it beats
  // the untiled best by more than 2 % (the timing noise of a few replays)
  if (best_ms < 1e30 && !best.res) {
    const BatchConfig base = best;
    const double base_ms = best_ms;
    best_ms = base_ms * 0.98;
    for (int C : {base.C, base.C / 2}) {
      if (C < 1) continue;
      for (int rt = 2; rt <= MAX_RTILES && (b->G * base.tpr) % rt == 0; rt *= 2)
        for (int div : {1, 2, 8, 32}) {
          const int top = std::max(1, b->count / div);
          if (div > 1 && top == b->count) continue;
          BatchConfig c = base;
          c.C = C;
          c.rtiles = rt;
          c.top = div == 1 ? 0 : top;
          kpm_status s_ = time_cfg(c);
          if (s_ != KPM_OK) return s_;
        }
    }
    if (best.rtiles == 1) best_ms = base_ms;  // no tiling beat the margin: best is base
  }
  if (best_ms >= 1e30) return fail(KPM_ECUDA, "no launchable batch configuration");
  b->cfg = best;
  b->tuned = true;
  b->last_ms = best_ms;
  cache_store(tune_key(b), best);
  return build_graph(b, best);
}

kpm_status kpm_batch_info(kpm_batch b, int* cluster, int* chunk, int* clusters_launched,
                          double* last_ms) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (cluster) *cluster = b->cfg.C;
  if (chunk) *chunk = b->cfg.chunk;
  if (clusters_launched) *clusters_launched = b->exec ? b->grid / std::max(1, b->exec_cfg.C) : 0;
  if (last_ms) {
    float ms = 0.f;
    if (b->exec && cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) *last_ms = ms;
    else {
      cudaGetLastError();
      *last_ms = b->last_ms;
    }
  }
  return KPM_OK;
}

kpm_status kpm_batch_set_config(kpm_batch b, int cluster, int chunk, int percent) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (cluster < 1 || cluster > 16 || (cluster & (cluster - 1)) || chunk < 1 || percent < 1 ||
      percent > 100)
    return fail(KPM_EINVAL, "bad batch configuration");
  b->cfg.C = cluster;
  b->cfg.chunk = chunk;
  b->cfg.frac = percent;
  return KPM_OK;
}

kpm_status kpm_batch_set_rtiles(kpm_batch b, int rtiles, int top) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (rtiles < 1 || rtiles > MAX_RTILES || (rtiles & (rtiles - 1)) || (b->G * b->cfg.tpr) % rtiles)
    return fail(KPM_EINVAL, "R-tiles must be 1, 2 or 4 and divide the chunks per row (" +
                                std::to_string(b->G * b->cfg.tpr) + ")");
  if (rtiles > 1 && b->cfg.res)
    return fail(KPM_EINVAL, "the resident form runs untiled instances (R-tiles 1)");
  b->cfg.rtiles = rtiles;
  b->cfg.top = top <= 0 || top >= b->count ? 0 : top;
  return KPM_OK;
}

kpm_status kpm_batch_set_chunk_bytes(kpm_batch b, int bytes) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (bytes != 32 && bytes != 16) return fail(KPM_EINVAL, "chunk bytes must be 16 or 32");
  const int tpr = bytes == 16 ? 2 : 1;
  if (tpr == 2 && !half_chunks_ok(b))
    return fail(KPM_EINVAL, "16-byte chunks take real FP32 vectors and stencil operators");
  if (tpr == 2 && b->cfg.res)
    return fail(KPM_EINVAL, "the resident form runs 32-byte chunks");
  if ((b->G * tpr) % b->cfg.rtiles)
    return fail(KPM_EINVAL, "the current R-tiles do not divide the chunks per row");
  b->cfg.tpr = tpr;
  return KPM_OK;
}

kpm_status kpm_batch_get_chunk_bytes(kpm_batch b, int* bytes, int* threads_per_row) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (bytes) *bytes = b->cfg.tpr == 2 ? 16 : (b->fp32 ? 32 : 16);
  if (threads_per_row) *threads_per_row = b->G * b->cfg.tpr;
  return KPM_OK;
}

kpm_status kpm_batch_set_resident(kpm_batch b, int resident) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (resident != 0 && resident != 1) return fail(KPM_EINVAL, "resident must be 0 or 1");
  if (resident && !b->handles[0]->stencil)
    return fail(KPM_EINVAL, "the resident form takes stencil operators only");
  if (resident && b->cfg.tpr != 1)
    return fail(KPM_EINVAL, "the resident form runs 32-byte chunks");
  b->cfg.res = resident ? FORM_RESIDENT : FORM_GLOBAL;
  if (resident) {
    b->cfg.rtiles = 1;
    b->cfg.top = 0;
  }
  return KPM_OK;
}

kpm_status kpm_batch_get_resident(kpm_batch b, int* resident, int* min_cluster) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (resident) *resident = b->cfg.res == FORM_RESIDENT;
  if (min_cluster) {
    KPM_CUDA(cudaSetDevice(b->device));
    *min_cluster = 0;
    if (b->handles[0]->stencil)
      for (int C = 1; C <= 16; C *= 2)
        if (max_clusters_res(b, C) > 0) {
          *min_cluster = C;
          break;
        }
  }
  return KPM_OK;
}

kpm_status kpm_batch_set_staged(kpm_batch b, int staged) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (staged != 0 && staged != 1) return fail(KPM_EINVAL, "staged must be 0 or 1");
  if (staged && !staged_ok(b))
    return fail(KPM_EINVAL, "the staged form takes stencil operators with rows of at most 32 chunks");
  if (staged && b->cfg.tpr != 1)
    return fail(KPM_EINVAL, "the staged form runs 32-byte chunks");
  if (staged) {
    b->cfg.res = FORM_STAGED;
    b->cfg.rtiles = 1;
    b->cfg.top = 0;
  } else if (b->cfg.res == FORM_STAGED) {
    b->cfg.res = FORM_GLOBAL;
  }
  return KPM_OK;
}

kpm_status kpm_batch_get_staged(kpm_batch b, int* staged, int* tile_rows, int* stages) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (staged) *staged = b->cfg.res == FORM_STAGED;
  const StgShape sh = stg_shape(b, b->cfg.chunk);
  if (tile_rows) *tile_rows = 1 << sh.Tl;
  if (stages) *stages = 1 << sh.Sl;
  return KPM_OK;
}

kpm_status kpm_batch_get_rtiles(kpm_batch b, int* rtiles, int* top, int* max_rtiles) {
  if (!b) return fail(KPM_EINVAL, "batch is NULL");
  if (rtiles) *rtiles = b->cfg.rtiles;
  if (top) *top = b->cfg.rtiles > 1 ? (b->cfg.top <= 0 ? b->count : b->cfg.top) : 0;
  if (max_rtiles) *max_rtiles = std::min(MAX_RTILES, b->G * b->cfg.tpr);
  return KPM_OK;
}

void kpm_batch_destroy(kpm_batch b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->d_pool) cudaFree(b->d_pool);
  if (b->d_tasks) cudaFree(b->d_tasks);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->ev[0]) cudaEventDestroy(b->ev[0]);
  if (b->ev[1]) cudaEventDestroy(b->ev[1]);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // extern "C"
