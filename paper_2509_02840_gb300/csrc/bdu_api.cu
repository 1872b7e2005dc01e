// Host side of the C ABI declared in include/bdu.h: handle lifecycle,
// argument validation, device memory, and the order of the kernels of one
// update (Sec. 3.2: project, reduce, compose).
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cublas_v2.h>

#include "bdu_internal.cuh"

namespace bdu {
namespace {
std::atomic<int> g_inject_site{BDU_INJECT_NONE};
std::atomic<long long> g_inject_value{0};
}  // namespace
Injection injection() { return Injection{g_inject_site.load(), g_inject_value.load()}; }

cudaError_t launch_project_nz(int precision, const void *X, int64_t ld, int nrow, int ncol,
                              const double *B, int64_t ldb, int r, double *U, int64_t ldu,
                              int32_t *nz_ws, cudaStream_t s);
}

using namespace bdu;

namespace {

// ---------------------------------------------------------------- allocator
std::atomic<bdu_alloc_fn> g_alloc{nullptr};
std::atomic<bdu_free_fn> g_free{nullptr};
std::atomic<void *> g_alloc_ctx{nullptr};

thread_local char t_create_err[512] = "";

struct Alloc {
  bdu_alloc_fn fa;
  bdu_free_fn ff;
  void *ctx;
  int device;
  void *get(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (fa) return fa(bytes, device, ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void *p) {
    if (!p) return;
    if (ff) ff(p, device, ctx);
    else cudaFree(p);
  }
};

}  // namespace

struct bdu_ctx {
  int64_t m, n, N;  // of the problem held: m >= n (the transpose of the caller's when tr)
  // The caller's m < n: A = Q L P^T with L lower bidiagonal is held as
  // A^T = P L^T Q^T, whose L^T is upper bidiagonal with the same d, e.  The
  // entry points swap Q and P, B and C, the sides of rotations and the
  // per-factor statistics; everything below works on the m >= n problem.
  bool tr = false;
  bdu_options opt;
  int device;
  cudaStream_t stream;
  bool own_stream;
  Alloc al;
  std::vector<void *> blocks;
  std::vector<size_t> block_bytes;
  // factorization
  void *Q, *P;   // FP64 or FP32 (opt.precision)
  double *band;  // band_doubles(m, n)
  // per-update workspace (grown on demand)
  int64_t rcap;
  double *dB, *dC, *U, *V;
  int32_t *nzB, *nzC;
  // rotation stream of one rank-1 column
  RotStream st;
  int *status;
  unsigned long long *counters;
  double *scratch64;  // for conversions in read (mixed form)
  // orthogonality control (mixed form)
  void *cublas;           // created on first use
  double *ortho_ws;       // 3*m+1 doubles
  double *rx_E, *rx_W;    // re-orthogonalization workspace (floats; reorth32_workspace), allocated on first use
  int64_t since_check;
  int64_t cols_since_reorth[2];  // rank-1 columns since the last unconditional step (Q, P)
  double ortho[2];        // last estimates for Q, P (-1 = none)
  // automatic check in flight: the two squared estimates land in probe_host
  // (pinned) and probe_ev marks their arrival; acted on once it has fired
  double *probe_host;
  cudaEvent_t probe_ev;
  bool probe_pending;
  int64_t reorth[2];
  // overlapped mixed form: two record buffers and two more streams
  bool ovl;
  RotStream stb[2];      // st == stb[cur]
  int cur;               // buffer of the most recent rank-1 column
  bool pend;             // that column's application to Q, P is not enqueued yet
  bool apply_ev_set[2];
  bool pipe_ok, pipe_failed;  // rank-r pipeline resources present / could not be made
  cudaStream_t sa;       // applications (lowest priority)
  cudaStream_t sc;       // projections' rotation and chases (highest priority)
  cudaEvent_t ev_call, ev_proj, ev_rot, ev_chase, ev_apply[2];
  // descriptor workspace of batched updates led by this handle, and a second
  // stream on which their small items' chases run beside the large ones'
  cudaStream_t batch_aux;
  void *batch_ws;
  size_t batch_ws_bytes;
  // the captured launch sequence of a plain update, replayed while the rank
  // and the buffers it reads are the same (null = none; g_off after a failed capture)
  cudaGraphExec_t gexec;
  int64_t g_r;
  const double *g_B, *g_C;
  double *g_U;
  int32_t *g_rec;      // the record buffer the graph writes (h->st.La)
  int64_t g_launches;  // kernels one replay launches
  int64_t g_reorth[2];  // re-orthogonalizations one replay performs
  int64_t g_cols[2], g_cols_after[2];  // re-orthogonalization cadence counters before / after
  bool g_off;
  // BHU (bdu_update_bhu): the compact representation and its workspace,
  // allocated on first use
  double *bhu_Y, *bhu_W, *bhu_SL, *bhu_SR, *bhu_ws, *bhu_G1, *bhu_G2, *bhu_vec;
  unsigned *bhu_cnt;
  int64_t bhu_updates;
  int64_t graph_replays;
  // apply variant per side (launch_apply), and whether the autotuner is still
  // to run after the next update
  int apply_var[2];
  bool tune_pending;
  int64_t tunings;
  // bookkeeping
  int64_t updates;
  int64_t launches;
  bool timing;
  // pending (start, stop, which) event triples; which: 0 project, 1 chase, 2 apply Q, 3 apply P
  struct Ev { cudaEvent_t a, b; int which; };
  std::vector<Ev> pending;
  double ms[4];
  int64_t timed_updates, apply_launches;
  bool poisoned;
  std::atomic<int> busy;
  char err[512];
};

namespace {

size_t esize(const bdu_ctx *h) { return h->opt.precision == BDU_FP64 ? sizeof(double) : sizeof(float); }

bdu_status fail(bdu_ctx *h, bdu_status code, const char *fmt, ...) {
  char *buf = h ? h->err : t_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  if (h && (code == BDU_ECUDA || code == BDU_ETIMEOUT || code == BDU_EINTERNAL)) h->poisoned = true;
  return code;
}

bdu_status cuda_fail(bdu_ctx *h, cudaError_t e, const char *what) {
  return fail(h, BDU_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dev_alloc(bdu_ctx *h, size_t bytes) {
  void *p = h->al.get(bytes);
  if (p) {
    h->blocks.push_back(p);
    h->block_bytes.push_back(bytes);
  }
  return p;
}

void dev_free(bdu_ctx *h, void *p) {
  if (!p) return;
  for (size_t i = 0; i < h->blocks.size(); i++)
    if (h->blocks[i] == p) {
      h->blocks[i] = h->blocks.back();
      h->blocks.pop_back();
      h->block_bytes[i] = h->block_bytes.back();
      h->block_bytes.pop_back();
      break;
    }
  h->al.put(p);
}

bool all_finite(const double *x, int64_t count) {
  for (int64_t i = 0; i < count; i++)
    if (!std::isfinite(x[i])) return false;
  return true;
}

struct Guard {
  bdu_ctx *h;
  bool ok;
  explicit Guard(bdu_ctx *hh) : h(hh), ok(false) {
    int expect = 0;
    ok = h->busy.compare_exchange_strong(expect, 1);
  }
  ~Guard() {
    if (ok) h->busy.store(0);
  }
};

bdu_status ensure_rank_workspace(bdu_ctx *h, int64_t r) {
  if (r <= h->rcap) return BDU_OK;
  double *dB = (double *)h->al.get(sizeof(double) * h->m * r);
  double *dC = (double *)h->al.get(sizeof(double) * h->n * r);
  double *U = (double *)h->al.get(sizeof(double) * h->m * r);
  double *V = (double *)h->al.get(sizeof(double) * h->n * r);
  int32_t *nzB = (int32_t *)h->al.get(sizeof(int32_t) * (h->m * r + r));
  int32_t *nzC = (int32_t *)h->al.get(sizeof(int32_t) * (h->n * r + r));
  if (!dB || !dC || !U || !V || !nzB || !nzC) {
    h->al.put(dB); h->al.put(dC); h->al.put(U); h->al.put(V); h->al.put(nzB); h->al.put(nzC);
    return fail(h, BDU_ENOMEM, "device allocation for a rank-%lld update failed", (long long)r);
  }
  dev_free(h, h->dB); dev_free(h, h->dC); dev_free(h, h->U); dev_free(h, h->V);
  dev_free(h, h->nzB); dev_free(h, h->nzC);
  const size_t sz[6] = {sizeof(double) * h->m * r, sizeof(double) * h->n * r, sizeof(double) * h->m * r,
                        sizeof(double) * h->n * r, sizeof(int32_t) * (h->m * r + r), sizeof(int32_t) * (h->n * r + r)};
  int q = 0;
  for (void *p : {(void *)dB, (void *)dC, (void *)U, (void *)V, (void *)nzB, (void *)nzC}) {
    h->blocks.push_back(p);
    h->block_bytes.push_back(sz[q++]);
  }
  h->dB = dB; h->dC = dC; h->U = U; h->V = V; h->nzB = nzB; h->nzC = nzC;
  h->rcap = r;
  return BDU_OK;
}

// Kernel-group timing: an event pair around each group, resolved at sync.
struct Timer {
  bdu_ctx *h;
  int which;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  Timer(bdu_ctx *hh, int w, cudaStream_t st = nullptr) : h(hh), which(w), s(st ? st : hh->stream) {
    if (!h->timing) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      a = b = nullptr;
      return;
    }
    cudaEventRecord(a, s);
  }
  ~Timer() {
    if (!a) return;
    cudaEventRecord(b, s);
    h->pending.push_back({a, b, which});
  }
};

void resolve_timers(bdu_ctx *h) {
  for (auto &ev : h->pending) {
    float t = 0.f;
    if (cudaEventSynchronize(ev.b) == cudaSuccess && cudaEventElapsedTime(&t, ev.a, ev.b) == cudaSuccess)
      h->ms[ev.which] += t;
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  cudaGetLastError();
  h->pending.clear();
}

bdu_status check_device_status(bdu_ctx *h) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronizing the handle's stream");
  if (st & ERR_STEPS) return fail(h, BDU_ETIMEOUT, "the bulge-chase engine exceeded its step budget");
  if (st & ERR_APPLY) return fail(h, BDU_ETIMEOUT, "a bounded wait of the rotation apply ran out");
  if (st & ERR_ROTVEC) return fail(h, BDU_ETIMEOUT, "a bounded wait of the vector rotation ran out");
  if (st & ERR_GEMM) return fail(h, BDU_ETIMEOUT, "a bounded wait of the re-orthogonalization GEMM ran out");
  if (st & ERR_BHU) return fail(h, BDU_ETIMEOUT, "a grid barrier of the BHU kernel ran out");
  if (st & ERR_RANGE) return fail(h, BDU_EINTERNAL, "a rotation record named a pair outside the vector");
  if (st) return fail(h, BDU_EINTERNAL, "device invariant check failed (status bits 0x%x)", st);
  return BDU_OK;
}

// Enqueues the estimate of ||X^T X - I||_2 for Q (which = 0) or P (which = 1):
// the power iteration, then a copy of the squared estimate to *dst.
cudaError_t enqueue_probe(bdu_ctx *h, int which, double *dst, cudaStream_t s) {
  const int k = (int)(which == 0 ? h->m : h->n);
  cudaError_t e = launch_ortho_probe(h->opt.precision, which == 0 ? h->Q : h->P, k, h->ortho_ws, 20, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, h->ortho_ws + 3 * k, sizeof(double), cudaMemcpyDeviceToHost, s);
  return e;
}

// ---- overlapped mixed form -------------------------------------------------
// SMs an overlapped apply leaves to the concurrent chase (its cluster).
constexpr int kChaseSMs = 16;

// Enqueues on the apply stream the application of record buffer buf to Q and
// P, after everything enqueued so far on the handle's stream (and after the
// event `after`, if given).  The buffer's chase descriptors are current.
bdu_status reorth_factor(bdu_ctx *h, int which, cudaStream_t s);

// Columns between unconditional steps for a factor of order k: FP32 rounding
// in the application moves ||X^T X - I||_2 by about 3e-8 sqrt(k) per rank-1
// column (measured for k = 64 .. 4096), and a step leaves ~1e-6, so every
// 100 / sqrt(k) columns keeps it near half the 1e-5 tolerance.
int auto_cadence(int64_t k) {
  const int c = (int)(100.0 / sqrt((double)(k > 1 ? k : 1)));
  return c > 1 ? c : 1;
}

// The mixed form's unconditional re-orthogonalization: one Newton-Schulz step
// on Q (P) behind the application of the first column and then of every
// reorth_every-th (automatic: auto_cadence of its order, or every column for a
// factor that the blocked tensor-core apply updates), enqueued on s.
bdu_status reorth_after_column(bdu_ctx *h, cudaStream_t s) {
  if (h->opt.precision != BDU_MIXED || h->opt.reorth_every == 0) return BDU_OK;
  for (int which = 0; which < 2; which++) {
    // The blocked apply's products drift the factor's column norms about ten
    // times as fast as rotation-by-rotation FP32 application (the tensor
    // cores' accumulation truncates toward zero); the step removes exactly
    // that symmetric part of the error, so it follows every column there.
    const int64_t dim = which == 0 ? h->m : h->n;
    // (the blocked apply: the variant chosen, or the library's rule for the order)
    const bool blocked = is_tc_variant(h->apply_var[which]) ||
                         (h->apply_var[which] == 0 && dim >= kBlockedFrom && h->st.tc_ws);
    const int every = h->opt.reorth_every > 0 ? h->opt.reorth_every : blocked ? 1 : auto_cadence(dim);
    if (++h->cols_since_reorth[which] < every && h->reorth[which] > 0) continue;
    h->cols_since_reorth[which] = 0;
    const bdu_status st = reorth_factor(h, which, s);
    if (st != BDU_OK) return st;
  }
  return BDU_OK;
}

bdu_status enqueue_apply(bdu_ctx *h, int buf, int sm_reserve, cudaEvent_t after = nullptr) {
  const int m = (int)h->m, n = (int)h->n;
  cudaError_t e = cudaEventRecord(h->ev_call, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->sa, h->ev_call, 0);
  if (e == cudaSuccess && after) e = cudaStreamWaitEvent(h->sa, after, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "ordering the apply stream");
  {
    Timer tm(h, 2, h->sa);
    e = launch_apply(h->opt.precision, h->Q, m, m, m, h->stb[buf], 0, m > n, h->sa, h->status, sm_reserve, true,
                     h->apply_var[0]);
    if (e != cudaSuccess) return cuda_fail(h, e, "apply to Q");
  }
  {
    Timer tm(h, 3, h->sa);
    e = launch_apply(h->opt.precision, h->P, n, n, n, h->stb[buf], 1, false, h->sa, h->status, sm_reserve, true,
                     h->apply_var[1]);
    if (e != cudaSuccess) return cuda_fail(h, e, "apply to P");
  }
  const bdu_status rs = reorth_after_column(h, h->sa);
  if (rs != BDU_OK) return rs;
  e = cudaEventRecord(h->ev_apply[buf], h->sa);
  if (e != cudaSuccess) return cuda_fail(h, e, "ordering the apply stream");
  h->apply_ev_set[buf] = true;
  h->launches += 2;
  if (h->timing) h->apply_launches += 2;
  return BDU_OK;
}

// Enqueues a deferred application, if any, and orders the handle's stream
// after it: afterwards Q and P are current for work on that stream.
bdu_status flush_apply(bdu_ctx *h) {
  if (!h->ovl || !h->pend) return BDU_OK;
  h->pend = false;
  bdu_status st = enqueue_apply(h, h->cur, 0);
  if (st != BDU_OK) return st;
  cudaError_t e = cudaStreamWaitEvent(h->stream, h->ev_apply[h->cur], 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "ordering after the apply stream");
  return BDU_OK;
}

// The same estimate, waited for.
bdu_status probe_factor(bdu_ctx *h, int which, double *est) {
  double acc = 0.0;
  bdu_status fs = flush_apply(h);
  if (fs != BDU_OK) return fs;
  cudaError_t e = enqueue_probe(h, which, &acc, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "orthogonality probe");
  *est = sqrt(acc);
  h->ortho[which] = *est;
  return BDU_OK;
}

// One Newton-Schulz step on Q (which = 0) or P, enqueued on stream s.
bdu_status reorth_factor(bdu_ctx *h, int which, cudaStream_t s) {
  const int64_t k = which == 0 ? h->m : h->n;
  if (!h->rx_E) {
    size_t ef = 0, wf = 0;
    reorth32_workspace(h->m, (int)h->m, &ef, &wf);  // Q's order is the larger
    h->rx_E = (double *)dev_alloc(h, sizeof(float) * ef);
    h->rx_W = (double *)dev_alloc(h, sizeof(float) * wf);
    if (!h->rx_E || !h->rx_W) {
      dev_free(h, h->rx_E); dev_free(h, h->rx_W);
      h->rx_E = h->rx_W = nullptr;
      return fail(h, BDU_ENOMEM, "re-orthogonalization workspace allocation failed");
    }
  }
  cudaError_t e = launch_reorth32((float *)(which == 0 ? h->Q : h->P), k, (int)k, (float *)h->rx_E, (float *)h->rx_W,
                                  h->status, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "re-orthogonalization");
  h->reorth[which]++;
  return BDU_OK;
}

// Acts on a finished automatic check: records both estimates and
// re-orthogonalizes a factor whose estimate exceeds reorth_tol.
bdu_status resolve_probe(bdu_ctx *h) {
  h->probe_pending = false;
  for (int which = 0; which < 2; which++) {
    const double est = sqrt(h->probe_host[which]);
    h->ortho[which] = est;
    if (h->opt.reorth_tol > 0.0 && est > h->opt.reorth_tol) {
      // overlapped with an application deferred: on the apply stream, between
      // the applications already enqueued and the next (the factor is then
      // re-orthogonalized at that point of its update sequence); otherwise
      // after all work on the handle's stream
      bdu_status st = BDU_OK;
      if (h->ovl && h->pend) {
        cudaError_t e = cudaEventRecord(h->ev_call, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->sa, h->ev_call, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "ordering the re-orthogonalization");
        st = reorth_factor(h, which, h->sa);
      } else {
        st = flush_apply(h);
        if (st == BDU_OK) st = reorth_factor(h, which, h->stream);
      }
      if (st != BDU_OK) return st;
    }
  }
  return BDU_OK;
}

// Waits for an automatic check still in flight and acts on it (at every call
// that synchronizes, so that what it returns reflects the check).
bdu_status settle_probe(bdu_ctx *h) {
  if (!h->probe_pending) return BDU_OK;
  cudaError_t e = cudaEventSynchronize(h->probe_ev);
  if (e != cudaSuccess) return cuda_fail(h, e, "orthogonality probe");
  return resolve_probe(h);
}

// Mixed form: every check_every updates, probe both factors.  The probe is
// only enqueued; its result is acted on by the first later update that finds
// it finished, or by the next synchronizing call, so that no update waits on
// the host for it.  A check falling due while one is in flight waits for it.
bdu_status maybe_reorth(bdu_ctx *h, int64_t r) {
  if (h->opt.precision != BDU_MIXED || h->opt.check_every <= 0) return BDU_OK;
  if (h->probe_pending) {
    cudaError_t q = cudaEventQuery(h->probe_ev);
    if (q == cudaSuccess) {
      bdu_status st = resolve_probe(h);
      if (st != BDU_OK) return st;
    } else if (q != cudaErrorNotReady) {
      return cuda_fail(h, q, "orthogonality probe");
    }
  }
  h->since_check += r;
  if (h->since_check < h->opt.check_every || h->probe_pending) return BDU_OK;
  h->since_check = 0;
  // overlapped with an application deferred: on the apply stream, behind the
  // latest enqueued application and everything on the handle's stream
  const cudaStream_t ps = (h->ovl && h->pend) ? h->sa : h->stream;
  cudaError_t e = cudaSuccess;
  if (ps != h->stream) {
    e = cudaEventRecord(h->ev_call, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ps, h->ev_call, 0);
  }
  if (e == cudaSuccess) e = enqueue_probe(h, 0, &h->probe_host[0], ps);
  if (e == cudaSuccess) e = enqueue_probe(h, 1, &h->probe_host[1], ps);
  if (e == cudaSuccess) e = cudaEventRecord(h->probe_ev, ps);
  if (e != cudaSuccess) return cuda_fail(h, e, "orthogonality probe");
  h->probe_pending = true;
  return BDU_OK;
}

// One overlapped rank-1 update (mixed form).  Streams: the handle's stream s
// (the caller's order), the chase stream sc and the apply stream sa.  With the
// previous column's application still deferred: on sa, project b and c with
// Q and P as they are before it; on sc, rotate the projections by that
// column's rotations (u = G^T Q^T b, v = H^T P^T c), then run this column's
// chase into the other record buffer; on sa, the previous column's
// application starts once the rotation is done, so that it runs beside the
// chase, which has the higher priority and is placed first.  s waits for the
// chase; this column's application is deferred in turn.
void drop_graph(bdu_ctx *h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
}

// ------------------------------------------------------------------ autotuner
// The apply variant of each side (launch_apply: the slab kernel's rows per
// block in the FP64 form, the register layout or the slab kernel in the mixed
// form) is picked by timing.  After the first update of a handle created with
// nb = 0 whose shape is not yet known, every candidate runs on a scratch copy
// of the factor with that update's rotation records (twice when a run takes
// under 2 ms, the faster counting), and the fastest candidate is kept (all
// candidates give identical results).  Choices are
// cached for the process per (GPU, form, order of the factor, SMs left to the
// apply) and, when the environment variable BDU_TUNE_FILE names a file, kept
// there as a JSON object {"key": variant, ...}: read on first use, rewritten
// after every new choice.
namespace tune {
std::mutex mu;
std::map<std::string, int> table;
bool loaded = false;

std::string key(const bdu_ctx *h, int dim, int sm_reserve) {
  cudaDeviceProp p{};
  cudaGetDeviceProperties(&p, h->device);
  char buf[512];
  snprintf(buf, sizeof buf, "%s|%s|%d|%d", p.name, h->opt.precision == BDU_FP64 ? "fp64" : "mixed", dim,
           sm_reserve);
  for (char *c = buf; *c; c++)
    if (*c == '"' || *c == '\\') *c = '_';
  return buf;
}

// caller holds mu
void load() {
  if (loaded) return;
  loaded = true;
  const char *path = getenv("BDU_TUNE_FILE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  std::string text;
  char chunk[4096];
  size_t got;
  while ((got = fread(chunk, 1, sizeof chunk, f)) > 0) text.append(chunk, got);
  fclose(f);
  size_t i = 0;
  while ((i = text.find('"', i)) != std::string::npos) {
    const size_t j = text.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string k = text.substr(i + 1, j - i - 1);
    const size_t c = text.find(':', j);
    if (c == std::string::npos) break;
    char *end = nullptr;
    const long v = strtol(text.c_str() + c + 1, &end, 10);
    if (end != text.c_str() + c + 1) table[k] = (int)v;
    i = end ? (size_t)(end - text.c_str()) : c + 1;
  }
}

// caller holds mu
void save() {
  const char *path = getenv("BDU_TUNE_FILE");
  if (!path || !*path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t k = 0;
  for (const auto &kv : table) fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < table.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}
}  // namespace tune

// Picks the apply variant of one side; the rotation records of the latest
// rank-1 column must be complete (the handle's stream synchronized) and not
// yet applied, or applied: only a scratch copy of the factor is touched.
bdu_status tune_side(bdu_ctx *h, int side, int sm_reserve) {
  const int m = (int)h->m, n = (int)h->n, dim = side == 0 ? m : n;
  const bool mixed = h->opt.precision == BDU_MIXED;
  if (mixed && dim >= kBlockedFrom && h->st.tc_ws) {
    h->apply_var[side] = 128;  // the fixed rule, not a timing (see kBlockedFrom)
    return BDU_OK;
  }
  const std::string k = tune::key(h, dim, sm_reserve);
  {
    std::lock_guard<std::mutex> lk(tune::mu);
    tune::load();
    auto it = tune::table.find(k);
    if (it != tune::table.end() && !(mixed && is_tc_variant(it->second))) {
      h->apply_var[side] = it->second;
      return BDU_OK;
    }
  }
  // candidates that round alike (FP64: slab heights; mixed: the FP32 register
  // layouts and the FP32 slab), so that the choice changes no result
  std::vector<int> cand;
  if (!mixed) {
    for (int R : {2, 4, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64}) cand.push_back(R);
  } else {
    for (int v = 1; v <= 4; v++) cand.push_back(v);
    cand.push_back(kSlabVariant);
  }
  const size_t bytes = esize(h) * (size_t)dim * dim;
  void *scratch = dev_alloc(h, bytes);
  if (!scratch) return BDU_OK;  // no room: keep the library's choice
  cudaStream_t s = h->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  int best = 0;
  float best_ms = 3.0e38f;
  void *X = side == 0 ? h->Q : h->P;
  for (size_t c = 0; c < cand.size() && ce == cudaSuccess; c++) {
    float ms = 3.0e38f;
    for (int rep = 0; rep < 2 && ce == cudaSuccess; rep++) {
      ce = cudaMemcpyAsync(scratch, X, bytes, cudaMemcpyDeviceToDevice, s);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
      if (ce != cudaSuccess) break;
      const cudaError_t le = launch_apply(h->opt.precision, scratch, dim, dim, dim, h->st, side, side == 0 && m > n, s,
                                          h->status, sm_reserve, false, cand[c]);
      if (le == cudaErrorNotSupported) {
        cudaGetLastError();
        break;
      }
      ce = le;
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float t = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
      if (ce == cudaSuccess && t < ms) ms = t;
      if (t > 2.0f) break;  // long enough to time once
    }
    if (ce == cudaSuccess && ms < best_ms) { best_ms = ms; best = cand[c]; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  dev_free(h, scratch);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "autotuning the apply");
  h->apply_var[side] = best;
  h->tunings++;
  std::lock_guard<std::mutex> lk(tune::mu);
  tune::table[k] = best;
  tune::save();
  return BDU_OK;
}

// After an update: runs the autotuner once the first update's records exist.
bdu_status maybe_tune(bdu_ctx *h) {
  if (!h->tune_pending || h->st.T <= 0) return BDU_OK;
  h->tune_pending = false;
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotuning the apply");
  const int reserve = h->ovl ? kChaseSMs : 0;
  bdu_status st = tune_side(h, 0, reserve);
  if (st == BDU_OK) st = tune_side(h, 1, reserve);
  drop_graph(h);  // captured with the previous variants
  return st;
}

bdu_status finish_update(bdu_ctx *h, int64_t r) {
  const bdu_status st = maybe_tune(h);
  return st != BDU_OK ? st : maybe_reorth(h, r);
}

// Copies d (n) and e (n-1) of the current bidiagonal from the band to the
// host (either may be null); synchronizes the handle's stream.
cudaError_t read_bidiagonal(bdu_ctx *h, double *d, double *e) {
  const int64_t m = h->m, n = h->n;
  std::vector<double> hb(band_doubles(m, n));
  cudaError_t ce = cudaMemcpyAsync(hb.data(), h->band, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return ce;
  BandPtrs hp = band_ptrs(hb.data(), m, n);
  if (d) {
    d[0] = hp.r1[1];
    for (int64_t i = 2; i <= n; i++) d[i - 1] = hp.dg[2][i];
  }
  if (e && n > 1) {
    e[0] = hp.r1[2];
    for (int64_t i = 2; i <= n - 1; i++) e[i - 1] = hp.dg[3][i];
  }
  return cudaSuccess;
}

bdu_status run_overlapped(bdu_ctx *h, const double *dB, const double *dC) {
  const int m = (int)h->m, n = (int)h->n;
  cudaStream_t s = h->stream, sa = h->sa, sc = h->sc;
  BandPtrs bp = band_ptrs(h->band, m, n);
  cudaError_t e = cudaEventRecord(h->ev_call, s);  // the previous chase and this update's inputs
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, h->ev_call, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "ordering the chase stream");
  if (h->timing) {
    h->timed_updates += 1;
    if (h->pending.size() > 4096) resolve_timers(h);
  }
  // this column's record buffer: free once the application two columns back
  // is done; cleared before the rotation, so that the chase follows it directly
  const int buf = h->pend ? (h->cur ^ 1) : h->cur;
  if (h->apply_ev_set[buf]) e = cudaStreamWaitEvent(sc, h->ev_apply[buf], 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->stb[buf].Ln, 0, sizeof(int32_t) * h->st.T, sc);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->stb[buf].Rn, 0, sizeof(int32_t) * h->st.T, sc);
  if (e != cudaSuccess) return cuda_fail(h, e, "staging a rank-1 column");
  if (h->pend) {
    const int prev = h->cur;
    e = cudaStreamWaitEvent(sa, h->ev_call, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "ordering the apply stream");
    {
      Timer tm(h, 0, sa);
      e = launch_project_nz(h->opt.precision, h->Q, m, m, m, dB, m, 1, h->U, m, h->nzB, sa);
      if (e == cudaSuccess) e = launch_project_nz(h->opt.precision, h->P, n, n, n, dC, n, 1, h->V, n, h->nzC, sa);
      if (e != cudaSuccess) return cuda_fail(h, e, "projection of b, c");
    }
    e = cudaEventRecord(h->ev_proj, sa);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, h->ev_proj, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "ordering after the projection");
    {
      Timer tm(h, 0, sc);
      e = launch_rotate_vectors(h->U, bp.u + 1, m, h->V, bp.v + 1, n, h->stb[prev], m > n, h->status, sc);
      if (e != cudaSuccess) return cuda_fail(h, e, "rotating the projections");
    }
    e = cudaEventRecord(h->ev_rot, sc);
    if (e != cudaSuccess) return cuda_fail(h, e, "ordering after the rotation");
    h->pend = false;
    bdu_status st = enqueue_apply(h, prev, kChaseSMs, h->ev_rot);
    if (st != BDU_OK) return st;
    h->launches += 5;
  } else {
    {
      Timer tm(h, 0, sc);
      e = launch_project_nz(h->opt.precision, h->Q, m, m, m, dB, m, 1, h->U, m, h->nzB, sc);
      if (e == cudaSuccess) e = launch_project_nz(h->opt.precision, h->P, n, n, n, dC, n, 1, h->V, n, h->nzC, sc);
      if (e != cudaSuccess) return cuda_fail(h, e, "projection of b, c");
    }
    e = cudaMemcpyAsync(bp.u + 1, h->U, sizeof(double) * m, cudaMemcpyDeviceToDevice, sc);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bp.v + 1, h->V, sizeof(double) * n, cudaMemcpyDeviceToDevice, sc);
    if (e != cudaSuccess) return cuda_fail(h, e, "staging a rank-1 column");
    h->launches += 4;
  }
  h->cur = buf;
  h->st = h->stb[buf];
  ChaseArgs a{};
  a.m = m; a.n = n; a.band = bp;
  a.rx = 0; a.Ux = nullptr; a.Vx = nullptr;
  a.st = h->st; a.status = h->status; a.counters = h->counters;
  a.fast = 1;
  a.engine = h->opt.engine;
  a.step_budget = h->opt.step_budget;
  {
    Timer tm(h, 1, sc);
    e = launch_chase(a, sc);
    if (e != cudaSuccess) return cuda_fail(h, e, "bulge-chase kernel");
  }
  // descriptors of this column's chases, for its application and for the
  // next column's vector rotation
  e = launch_chase_descriptors(h->st, 0, sc);
  if (e == cudaSuccess) e = launch_chase_descriptors(h->st, 1, sc);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_chase, sc);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_chase, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "chase descriptors");
  h->launches += 3;
  h->pend = true;
  h->updates++;
  return finish_update(h, 1);
}

// One update with B, C already in device memory.
bool alloc_records(bdu_ctx *h, RotStream &r, int T, int cap, int64_t m, bool mixed);

// Resources of the rank-r pipeline: a second record buffer, a chase stream of
// the greatest priority and an apply stream of the least (so that, when a
// column's application and the next column's chase become ready together, the
// chase's cluster is placed first), and events.  Made on the first rank-r
// update; false when they cannot be (the update then runs column by column).
bool ensure_pipeline(bdu_ctx *h) {
  if (h->pipe_ok) return true;
  if (h->pipe_failed) return false;
  h->pipe_failed = true;
  if (!h->stb[1].La) {
    h->stb[0] = h->st;
    h->cur = 0;
    const bool got = alloc_records(h, h->stb[1], h->st.T, h->st.cap, h->m, h->opt.precision == BDU_MIXED);
    h->stb[1].tc_ws = h->st.tc_ws;  // the applications of the two buffers run on one stream
    h->stb[1].tc_ws_bytes = h->st.tc_ws_bytes;
    if (!got) {
      for (void *p : {(void *)h->stb[1].Lc, (void *)h->stb[1].Ls, (void *)h->stb[1].Rc, (void *)h->stb[1].Rs,
                      (void *)h->stb[1].La, (void *)h->stb[1].Ra, (void *)h->stb[1].Ln, (void *)h->stb[1].Rn,
                      (void *)h->stb[1].Sc, (void *)h->stb[1].Ss, (void *)h->stb[1].Sa, (void *)h->stb[1].Sn,
                      (void *)h->stb[1].Lf, (void *)h->stb[1].Rf, (void *)h->stb[1].Sf, (void *)h->stb[1].Lm,
                      (void *)h->stb[1].Rm})
        dev_free(h, p);
      h->stb[1] = RotStream{};
      return false;
    }
  }
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (!h->sa && cudaStreamCreateWithPriority(&h->sa, cudaStreamNonBlocking, least) != cudaSuccess) h->sa = nullptr;
  if (!h->sc && cudaStreamCreateWithPriority(&h->sc, cudaStreamNonBlocking, greatest) != cudaSuccess) h->sc = nullptr;
  for (cudaEvent_t *ev : {&h->ev_call, &h->ev_chase, &h->ev_apply[0], &h->ev_apply[1]})
    if (!*ev && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) *ev = nullptr;
  if (!h->sa || !h->sc || !h->ev_call || !h->ev_chase || !h->ev_apply[0] || !h->ev_apply[1]) {
    cudaGetLastError();
    return false;
  }
  h->pipe_failed = false;
  h->pipe_ok = true;
  return true;
}

// The columns of a rank-r update, pipelined: column k's chase runs on the
// chase stream while column k-1 is applied to Q and P on the apply stream.
// The later columns' projections are rotated inside the chases (U(:, k+1:r),
// V(:, k+1:r)), so no column waits for an earlier column's application, and
// the results are those of the column-by-column order.  Record buffers
// alternate; a buffer is reused only after its column's application.
bdu_status enqueue_columns_pipelined(bdu_ctx *h, int64_t r) {
  const int m = (int)h->m, n = (int)h->n;
  cudaStream_t s = h->stream, sc = h->sc, sa = h->sa;
  BandPtrs bp = band_ptrs(h->band, m, n);
  cudaError_t e = cudaEventRecord(h->ev_call, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, h->ev_call, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sa, h->ev_call, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "ordering the rank-r pipeline");
  // Column k-1's application is enqueued once column k is staged, so that it
  // and column k's chase become ready together and the chase (on the stream
  // of greater priority) is placed first; the application leaves it SMs.
  bool desc_ready = false;  // set below, before the first application
  auto enqueue_apply_of = [&](int buf, int reserve) -> bdu_status {
    cudaError_t ee = cudaEventRecord(h->ev_chase, sc);
    if (ee == cudaSuccess) ee = cudaStreamWaitEvent(sa, h->ev_chase, 0);
    if (ee != cudaSuccess) return cuda_fail(h, ee, "ordering the rank-r pipeline");
    {
      Timer tm(h, 2, sa);
      ee = launch_apply(h->opt.precision, h->Q, m, m, m, h->stb[buf], 0, m > n, sa, h->status, reserve, desc_ready,
                        h->apply_var[0]);
      if (ee != cudaSuccess) return cuda_fail(h, ee, "apply to Q");
    }
    {
      Timer tm(h, 3, sa);
      ee = launch_apply(h->opt.precision, h->P, n, n, n, h->stb[buf], 1, false, sa, h->status, reserve, desc_ready,
                        h->apply_var[1]);
      if (ee != cudaSuccess) return cuda_fail(h, ee, "apply to P");
    }
    const bdu_status rs = reorth_after_column(h, sa);
    if (rs != BDU_OK) return rs;
    ee = cudaEventRecord(h->ev_apply[buf], sa);
    if (ee != cudaSuccess) return cuda_fail(h, ee, "ordering the rank-r pipeline");
    h->launches += 2;
    if (h->timing) h->apply_launches += 2;
    return BDU_OK;
  };
  // Mixed form: the later columns' projections are rotated by each column's
  // rotations after its chase, all at once (one block per vector, FP32 like
  // the application to Q and P), instead of inside the chase, where they
  // lengthened every step; the chase descriptors this needs also serve the
  // applications.  The FP64 form rotates them inside the chase (exact order).
  const bool after = h->opt.precision == BDU_MIXED && rotate_vectors_supported(m, n);
  desc_ready = after;
  int b = h->cur;
  for (int64_t k = 0; k < r; k++) {
    b ^= 1;
    RotStream &sb = h->stb[b];
    // this buffer's previous column (k-2) is applied before it is reused
    // (earlier calls' applications are behind the caller's stream already)
    if (k >= 2) e = cudaStreamWaitEvent(sc, h->ev_apply[b], 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "pipelined column: waiting for its record buffer");
    e = cudaMemcpyAsync(bp.u + 1, h->U + k * m, sizeof(double) * m, cudaMemcpyDeviceToDevice, sc);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bp.v + 1, h->V + k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, sc);
    if (e != cudaSuccess) return cuda_fail(h, e, "pipelined column: staging u, v");
    e = cudaMemsetAsync(sb.Ln, 0, sizeof(int32_t) * sb.T, sc);
    if (e == cudaSuccess) e = cudaMemsetAsync(sb.Rn, 0, sizeof(int32_t) * sb.T, sc);
    if (e != cudaSuccess) return cuda_fail(h, e, "pipelined column: clearing the record counts");
    if (k > 0) {
      const bdu_status st = enqueue_apply_of(b ^ 1, kChaseSMs);
      if (st != BDU_OK) return st;
    }
    ChaseArgs a{};
    a.m = m; a.n = n; a.band = bp;
    a.rx = after ? 0 : (int)(r - k - 1);
    a.Ux = a.rx > 0 ? h->U + (k + 1) * m : nullptr;
    a.Vx = a.rx > 0 ? h->V + (k + 1) * n : nullptr;
    a.st = sb; a.status = h->status; a.counters = h->counters;
    a.fast = (h->opt.precision == BDU_MIXED) ? 1 : 0;
    a.engine = h->opt.engine;
    a.step_budget = h->opt.step_budget;
    {
      Timer tm(h, 1, sc);
      e = launch_chase(a, sc);
      if (e != cudaSuccess) return cuda_fail(h, e, "bulge-chase kernel");
    }
    h->launches += 1;
    if (after) {
      e = launch_chase_descriptors(sb, 0, sc);
      if (e == cudaSuccess) e = launch_chase_descriptors(sb, 1, sc);
      const int later = (int)(r - k - 1);
      if (e == cudaSuccess && later > 0)
        e = launch_rotate_vector_sets(h->U + (k + 1) * m, h->U + (k + 1) * m, m, later, m, h->V + (k + 1) * n,
                                      h->V + (k + 1) * n, n, later, n, sb, m > n, h->status, sc);
      if (e != cudaSuccess) return cuda_fail(h, e, "rotating the later projections");
      h->launches += later > 0 ? 3 : 2;
    }
    h->updates++;
  }
  const bdu_status st = enqueue_apply_of(b, 0);
  if (st != BDU_OK) return st;
  // the caller's stream continues after the last application (which follows
  // the last chase on the apply stream); later work ordered after that stream
  // needs no wait on the buffers' events, which may have been recorded inside
  // a graph capture and cannot be waited on outside it
  e = cudaStreamWaitEvent(s, h->ev_apply[b], 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "ordering the rank-r pipeline");
  h->apply_ev_set[0] = h->apply_ev_set[1] = false;
  h->cur = b;
  h->st = h->stb[b];
  return BDU_OK;
}

// Enqueues the launches of a plain update (every rank-1 column in turn).
bdu_status enqueue_update(bdu_ctx *h, const double *dB, const double *dC, int64_t r) {
  const int m = (int)h->m, n = (int)h->n;
  cudaStream_t s = h->stream;
  cudaError_t e;
  if (h->timing) {
    h->timed_updates += r;
    if (h->pending.size() > 4096) resolve_timers(h);
  }
  // K1: U = Q^T B, V = P^T C with the current factors
  {
    Timer tm(h, 0);
    e = launch_project_nz(h->opt.precision, h->Q, m, m, m, dB, m, (int)r, h->U, m, h->nzB, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "projection of B");
    e = launch_project_nz(h->opt.precision, h->P, n, n, n, dC, n, (int)r, h->V, n, h->nzC, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "projection of C");
    h->launches += 4;
  }
  if (r > 1 && ensure_pipeline(h)) return enqueue_columns_pipelined(h, r);
  BandPtrs bp = band_ptrs(h->band, m, n);
  for (int64_t k = 0; k < r; k++) {
    // u = U(:,k), v = V(:,k) (1-based in the band buffer)
    e = cudaMemcpyAsync(bp.u + 1, h->U + k * m, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bp.v + 1, h->V + k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->st.Ln, 0, sizeof(int32_t) * h->st.T, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->st.Rn, 0, sizeof(int32_t) * h->st.T, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "staging a rank-1 column");
    // (mixed form: the later projections are rotated after the chase, as in
    // the pipelined path)
    const bool after = h->opt.precision == BDU_MIXED && r > 1 && rotate_vectors_supported(m, n);
    ChaseArgs a{};
    a.m = m; a.n = n; a.band = bp;
    a.rx = after ? 0 : (int)(r - k - 1);
    a.Ux = a.rx > 0 ? h->U + (k + 1) * m : nullptr;
    a.Vx = a.rx > 0 ? h->V + (k + 1) * n : nullptr;
    a.st = h->st; a.status = h->status; a.counters = h->counters;
    a.fast = (h->opt.precision == BDU_MIXED) ? 1 : 0;
    a.engine = h->opt.engine;
    a.step_budget = h->opt.step_budget;
    {
      Timer tm(h, 1);
      e = launch_chase(a, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "bulge-chase kernel");
    }
    if (after && k + 1 < r) {
      const int later = (int)(r - k - 1);
      e = launch_chase_descriptors(h->st, 0, s);
      if (e == cudaSuccess) e = launch_chase_descriptors(h->st, 1, s);
      if (e == cudaSuccess)
        e = launch_rotate_vector_sets(h->U + (k + 1) * m, h->U + (k + 1) * m, m, later, m, h->V + (k + 1) * n,
                                      h->V + (k + 1) * n, n, later, n, h->st, m > n, h->status, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "rotating the later projections");
      h->launches += 3;
    }
    // K3: Q <- Q prod G^T, P <- P prod H
    {
      Timer tm(h, 2);
      e = launch_apply(h->opt.precision, h->Q, m, m, m, h->st, 0, m > n, s, h->status, 0, false, h->apply_var[0]);
      if (e != cudaSuccess) return cuda_fail(h, e, "apply to Q");
    }
    {
      Timer tm(h, 3);
      e = launch_apply(h->opt.precision, h->P, n, n, n, h->st, 1, false, s, h->status, 0, false, h->apply_var[1]);
      if (e != cudaSuccess) return cuda_fail(h, e, "apply to P");
    }
    const bdu_status rs = reorth_after_column(h, s);
    if (rs != BDU_OK) return rs;
    h->launches += 3;
    if (h->timing) h->apply_launches += 2;
    h->updates++;
  }
  return BDU_OK;
}

bdu_status run_update(bdu_ctx *h, const double *dB, const double *dC, int64_t r) {
  if (h->ovl && r == 1) return run_overlapped(h, dB, dC);
  bdu_status fs = flush_apply(h);
  if (fs != BDU_OK) return fs;
  if (!h->opt.graphs || h->g_off || h->timing) {
    fs = enqueue_update(h, dB, dC, r);
    return fs != BDU_OK ? fs : finish_update(h, r);
  }
  cudaStream_t s = h->stream;
  if (h->gexec && h->g_r == r && h->g_B == dB && h->g_C == dC && h->g_U == h->U && h->g_rec == h->st.La &&
      h->g_cols[0] == h->cols_since_reorth[0] && h->g_cols[1] == h->cols_since_reorth[1] &&
      (h->reorth[0] > 0) == (h->g_cols_after[0] >= 0) && (h->reorth[1] > 0) == (h->g_cols_after[1] >= 0)) {
    const cudaError_t e = cudaGraphLaunch(h->gexec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "replaying the update graph");
    h->launches += h->g_launches;
    h->reorth[0] += h->g_reorth[0];
    h->reorth[1] += h->g_reorth[1];
    h->cols_since_reorth[0] = h->g_cols_after[0] >= 0 ? h->g_cols_after[0] : -1 - h->g_cols_after[0];
    h->cols_since_reorth[1] = h->g_cols_after[1] >= 0 ? h->g_cols_after[1] : -1 - h->g_cols_after[1];
    h->updates += r;
    h->graph_replays++;
    return finish_update(h, r);
  }
  // capture this rank's launch sequence, then run it
  drop_graph(h);
  const int64_t l0 = h->launches, u0 = h->updates, q0 = h->reorth[0], p0 = h->reorth[1];
  const int64_t c0 = h->cols_since_reorth[0], c1 = h->cols_since_reorth[1];
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->g_off = true;
    fs = enqueue_update(h, dB, dC, r);
    return fs != BDU_OK ? fs : finish_update(h, r);
  }
  fs = enqueue_update(h, dB, dC, r);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  cudaGraphExec_t ex = nullptr;
  if (fs == BDU_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (g) cudaGraphDestroy(g);
  if (fs != BDU_OK || e != cudaSuccess) {
    // not capturable here: launch separately from now on
    cudaGetLastError();
    if (ex) cudaGraphExecDestroy(ex);
    h->g_off = true;
    h->poisoned = false;
    h->launches = l0;
    h->updates = u0;
    h->reorth[0] = q0;
    h->reorth[1] = p0;
    h->cols_since_reorth[0] = c0;
    h->cols_since_reorth[1] = c1;
    fs = enqueue_update(h, dB, dC, r);
    return fs != BDU_OK ? fs : finish_update(h, r);
  }
  h->gexec = ex;
  h->g_r = r; h->g_B = dB; h->g_C = dC; h->g_U = h->U; h->g_rec = h->st.La;
  h->g_launches = h->launches - l0;
  h->g_reorth[0] = h->reorth[0] - q0;
  h->g_reorth[1] = h->reorth[1] - p0;
  // counters as the call found and left them; the sign of the latter records
  // whether the factor had been re-orthogonalized before the call (which
  // changes the first-column rule), so a replay needs the same
  h->g_cols[0] = c0; h->g_cols[1] = c1;
  h->g_cols_after[0] = q0 > 0 ? h->cols_since_reorth[0] : -1 - h->cols_since_reorth[0];
  h->g_cols_after[1] = p0 > 0 ? h->cols_since_reorth[1] : -1 - h->cols_since_reorth[1];
  e = cudaGraphLaunch(ex, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "launching the update graph");
  return finish_update(h, r);
}

// Allocates one buffer of rotation records; false if an allocation failed.
// The FP64 form keeps (c, s) in FP64; the mixed form keeps only their FP32
// copies (what its FP32 factors are rotated with) and the chase descriptors.
// Padded: the kernels that stream records read whole 16-byte units.
bool alloc_records(bdu_ctx *h, RotStream &r, int T, int cap, int64_t m, bool mixed) {
  const size_t tc = (size_t)T * cap;
  r.T = T; r.cap = cap; r.p1 = (int)(h->N - 1);
  if (!mixed) {
    r.Lc = (double *)dev_alloc(h, sizeof(double) * (tc + 2));
    r.Ls = (double *)dev_alloc(h, sizeof(double) * (tc + 2));
    r.Rc = (double *)dev_alloc(h, sizeof(double) * (tc + 2));
    r.Rs = (double *)dev_alloc(h, sizeof(double) * (tc + 2));
  }
  r.La = (int32_t *)dev_alloc(h, sizeof(int32_t) * (tc + 4));
  r.Ra = (int32_t *)dev_alloc(h, sizeof(int32_t) * (tc + 4));
  r.Ln = (int32_t *)dev_alloc(h, sizeof(int32_t) * (T + 1));
  r.Rn = (int32_t *)dev_alloc(h, sizeof(int32_t) * (T + 1));
  r.Sc = (double *)dev_alloc(h, sizeof(double) * (m + 1));
  r.Ss = (double *)dev_alloc(h, sizeof(double) * (m + 1));
  r.Sa = (int32_t *)dev_alloc(h, sizeof(int32_t) * (m + 1));
  r.Sn = (int32_t *)dev_alloc(h, sizeof(int32_t) * 4);
  bool ok = (mixed || (r.Lc && r.Ls && r.Rc && r.Rs)) && r.La && r.Ra && r.Ln && r.Rn && r.Sc && r.Ss && r.Sa && r.Sn;
  if (mixed) {
    r.Lf = (float2 *)dev_alloc(h, sizeof(float2) * (tc + 2));
    r.Rf = (float2 *)dev_alloc(h, sizeof(float2) * (tc + 2));
    r.Sf = (float2 *)dev_alloc(h, sizeof(float2) * (m + 1));
    r.Lm = (int4 *)dev_alloc(h, sizeof(int4) * (T + 1));
    r.Rm = (int4 *)dev_alloc(h, sizeof(int4) * (T + 1));
    ok = ok && r.Lf && r.Rf && r.Sf && r.Lm && r.Rm;
  }
  return ok;
}

struct BatchGuard {
  std::vector<bdu_ctx *> held;
  ~BatchGuard() {
    for (bdu_ctx *h : held) h->busy.store(0);
  }
};

}  // namespace

extern "C" {

void bdu_default_options(bdu_options *opt) {
  if (!opt) return;
  opt->precision = BDU_FP64;
  opt->nb = 0;
  opt->reorth_tol = 5e-6;
  opt->check_every = 10;
  opt->cuda_stream = nullptr;
  opt->device = 0;
  opt->engine = 0;
  opt->overlap = 0;
  opt->graphs = 1;
  opt->step_budget = 0;
  opt->reorth_every = -1;
}

int bdu_version(void) { return 100; }

void bdu_set_allocator(bdu_alloc_fn alloc, bdu_free_fn release, void *ctx) {
  g_alloc.store(alloc);
  g_free.store(release);
  g_alloc_ctx.store(ctx);
}

const char *bdu_last_error(bdu_handle h) { return h ? h->err : t_create_err; }

void bdu_destroy(bdu_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->sa) cudaStreamSynchronize(h->sa);
  if (h->sc) cudaStreamSynchronize(h->sc);
  if (h->batch_aux) cudaStreamSynchronize(h->batch_aux);
  resolve_timers(h);
  drop_graph(h);
  if (h->cublas) cublasDestroy((cublasHandle_t)h->cublas);
  if (h->probe_ev) cudaEventDestroy(h->probe_ev);
  for (cudaEvent_t ev : {h->ev_call, h->ev_proj, h->ev_rot, h->ev_chase, h->ev_apply[0], h->ev_apply[1]})
    if (ev) cudaEventDestroy(ev);
  if (h->sa) cudaStreamDestroy(h->sa);
  if (h->batch_aux) cudaStreamDestroy(h->batch_aux);
  if (h->sc) cudaStreamDestroy(h->sc);
  if (h->probe_host) cudaFreeHost(h->probe_host);
  for (void *p : h->blocks) h->al.put(p);
  h->blocks.clear();
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

bdu_status bdu_create(bdu_handle *out, int64_t m, int64_t n, const double *Q, const double *d,
                      const double *e, const double *P, const bdu_options *opt) {
  if (!out) return fail(nullptr, BDU_EINVAL, "bdu_create: output handle pointer is NULL");
  *out = nullptr;
  if (n < 1 || m < 1) return fail(nullptr, BDU_EINVAL, "bdu_create: need m, n >= 1 (m=%lld n=%lld)", (long long)m, (long long)n);
  if (m < n) {
    // the transposed problem: A^T = P L^T Q^T (n x m, upper bidiagonal L^T)
    const bdu_status st = bdu_create(out, n, m, P, d, e, Q, opt);
    if (st == BDU_OK) (*out)->tr = true;
    return st;
  }
  if (m > (1LL << 20)) return fail(nullptr, BDU_EINVAL, "bdu_create: m=%lld exceeds the supported 2^20", (long long)m);
  if (!Q || !d || !P || (n > 1 && !e)) return fail(nullptr, BDU_EINVAL, "bdu_create: NULL input pointer");
  bdu_options o;
  bdu_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != BDU_FP64 && o.precision != BDU_MIXED)
    return fail(nullptr, BDU_EINVAL, "bdu_create: unknown precision %d", o.precision);
  if (o.engine < 0 || o.engine > 2)
    return fail(nullptr, BDU_EINVAL, "bdu_create: unknown engine %d", o.engine);
  if (o.step_budget < 0) return fail(nullptr, BDU_EINVAL, "bdu_create: negative step budget");
  if (o.reorth_every < -1) return fail(nullptr, BDU_EINVAL, "bdu_create: reorth_every below -1");
  if (o.precision == BDU_FP64 ? (o.nb < 0 || o.nb > 64 || (o.nb & 1))
                               : (o.nb < 0 || (o.nb > kSlabVariant && !is_tc_variant(o.nb))))
    return fail(nullptr, BDU_EINVAL, "bdu_create: unknown apply variant nb=%d", o.nb);
  if (!all_finite(Q, m * m) || !all_finite(P, n * n) || !all_finite(d, n) || (n > 1 && !all_finite(e, n - 1)))
    return fail(nullptr, BDU_EINVAL, "bdu_create: non-finite value in Q, d, e or P");

  bdu_ctx *h = new (std::nothrow) bdu_ctx();
  if (!h) return fail(nullptr, BDU_ENOMEM, "bdu_create: host allocation failed");
  h->m = m; h->n = n; h->N = (m > n) ? n + 1 : n;
  h->opt = o; h->device = o.device;
  h->apply_var[0] = h->apply_var[1] = o.nb;
  h->tune_pending = o.nb == 0;
  h->busy.store(0);
  h->al = Alloc{g_alloc.load(), g_free.load(), g_alloc_ctx.load(), o.device};
  cudaError_t ce = cudaSetDevice(o.device);
  if (ce != cudaSuccess) {
    fail(nullptr, BDU_ECUDA, "cudaSetDevice(%d): %s", o.device, cudaGetErrorString(ce));
    delete h;
    return BDU_ECUDA;
  }
  if (o.cuda_stream) {
    h->stream = (cudaStream_t)o.cuda_stream;
    h->own_stream = false;
  } else {
    ce = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
      fail(nullptr, BDU_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(ce));
      delete h;
      return BDU_ECUDA;
    }
    h->own_stream = true;
  }
  const size_t es = esize(h);
  const int T = num_tasks(m, n), cap = task_cap(n);
  h->Q = dev_alloc(h, es * m * m);
  h->P = dev_alloc(h, es * n * n);
  h->band = (double *)dev_alloc(h, sizeof(double) * band_doubles(m, n));
  const bool mixed = o.precision == BDU_MIXED;
  bool rec_ok = alloc_records(h, h->st, T, cap, m, mixed);
  if (mixed && (m >= kBlockedFrom || is_tc_variant(o.nb))) {
    // the blocked tensor-core apply's workspace, for every block order and both
    // factors (factors below kBlockedFrom take it only when asked for: nb)
    size_t tcb = 0;
    for (int nb : {64, 96, 128}) tcb = std::max(tcb, tc_workspace_bytes((int)m, T, nb));
    h->st.tc_ws = dev_alloc(h, tcb);
    h->st.tc_ws_bytes = h->st.tc_ws ? tcb : 0;
    rec_ok = rec_ok && h->st.tc_ws;
  }
  h->ovl = mixed && o.overlap != 0 && rotate_vectors_supported((int)m, (int)n);
  if (h->ovl) {
    h->stb[0] = h->st;
    rec_ok = rec_ok && alloc_records(h, h->stb[1], T, cap, m, mixed);
    h->stb[1].tc_ws = h->st.tc_ws;  // the applications of the two buffers never overlap
    h->stb[1].tc_ws_bytes = h->st.tc_ws_bytes;
    // The chase's thread-block cluster needs 16 free SMs of one GPC: its
    // stream outranks the application's, so that when both become ready the
    // chase is placed first and the application fills the other SMs.
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (cudaStreamCreateWithPriority(&h->sa, cudaStreamNonBlocking, least) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->sc, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_call, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_proj, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_rot, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_chase, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_apply[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_apply[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      fail(nullptr, BDU_ENOMEM, "bdu_create: stream or event creation failed");
      bdu_destroy(h);
      return BDU_ENOMEM;
    }
  }
  h->status = (int *)dev_alloc(h, sizeof(int) * 4);
  h->counters = (unsigned long long *)dev_alloc(h, sizeof(unsigned long long) * 16);
  h->ortho[0] = h->ortho[1] = -1.0;
  h->ortho_ws = (double *)dev_alloc(h, sizeof(double) * (3 * m + 8));
  if (o.precision == BDU_MIXED) {
    h->scratch64 = (double *)dev_alloc(h, sizeof(double) * m * m);
    if (cudaHostAlloc((void **)&h->probe_host, 2 * sizeof(double), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->probe_ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      fail(nullptr, BDU_ENOMEM, "bdu_create: pinned host cell or event creation failed");
      bdu_destroy(h);
      return BDU_ENOMEM;
    }
  }
  bool ok = h->Q && h->P && h->band && rec_ok && h->status && h->counters && h->ortho_ws &&
            (o.precision == BDU_FP64 || h->scratch64);
  if (!ok) {
    fail(nullptr, BDU_ENOMEM, "bdu_create: device allocation failed (m=%lld n=%lld)", (long long)m, (long long)n);
    bdu_destroy(h);
    return BDU_ENOMEM;
  }
  if (ensure_rank_workspace(h, 1) != BDU_OK) {
    fail(nullptr, BDU_ENOMEM, "bdu_create: device allocation failed (workspace)");
    bdu_destroy(h);
    return BDU_ENOMEM;
  }
  // band: diagonal d, superdiagonal e; row 1 kept densely
  const int64_t nb = band_doubles(m, n);
  std::vector<double> hb(nb, 0.0);
  BandPtrs hp = band_ptrs(hb.data(), m, n);
  hp.r1[1] = d[0];
  if (n > 1) hp.r1[2] = e[0];
  for (int64_t i = 2; i <= n; i++) hp.dg[2][i] = d[i - 1];
  for (int64_t i = 2; i <= n - 1; i++) hp.dg[3][i] = e[i - 1];
  ce = cudaMemcpyAsync(h->band, hb.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess) {
    if (o.precision == BDU_FP64) {
      ce = cudaMemcpyAsync(h->Q, Q, sizeof(double) * m * m, cudaMemcpyHostToDevice, h->stream);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h->P, P, sizeof(double) * n * n, cudaMemcpyHostToDevice, h->stream);
    } else {
      ce = cudaMemcpyAsync(h->scratch64, Q, sizeof(double) * m * m, cudaMemcpyHostToDevice, h->stream);
      if (ce == cudaSuccess) ce = launch_convert_f64_to_f32(h->scratch64, (float *)h->Q, m * m, h->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h->scratch64, P, sizeof(double) * n * n, cudaMemcpyHostToDevice, h->stream);
      if (ce == cudaSuccess) ce = launch_convert_f64_to_f32(h->scratch64, (float *)h->P, n * n, h->stream);
    }
  }
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->counters, 0, sizeof(unsigned long long) * 16, h->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->st.Sn, 0, sizeof(int32_t) * 4, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) {
    fail(nullptr, BDU_ECUDA, "bdu_create: %s", cudaGetErrorString(ce));
    bdu_destroy(h);
    return BDU_ECUDA;
  }
  h->err[0] = 0;
  *out = h;
  return BDU_OK;
}

static bdu_status update_common(bdu_handle h, const double *B, const double *C, int64_t r, bool host) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (h->poisoned) return fail(h, BDU_EPOISONED, "handle poisoned by an earlier failure: %s", h->err);
  if (r < 0) return fail(h, BDU_EINVAL, "negative rank %lld", (long long)r);
  if (r == 0) return BDU_OK;
  if (!B || !C) return fail(h, BDU_EINVAL, "NULL update pointer");
  if (r > 4096) return fail(h, BDU_EINVAL, "rank %lld exceeds 4096", (long long)r);
  if (host && (!all_finite(B, h->m * r) || !all_finite(C, h->n * r)))
    return fail(h, BDU_EINVAL, "non-finite value in B or C");
  cudaError_t ce = cudaSetDevice(h->device);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaSetDevice");
  bdu_status st = ensure_rank_workspace(h, r);
  if (st != BDU_OK) return st;
  const double *dB = B, *dC = C;
  if (host) {
    ce = cudaMemcpyAsync(h->dB, B, sizeof(double) * h->m * r, cudaMemcpyHostToDevice, h->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h->dC, C, sizeof(double) * h->n * r, cudaMemcpyHostToDevice, h->stream);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "copying B, C to the device");
    dB = h->dB; dC = h->dC;
  }
  return run_update(h, dB, dC, r);
}

bdu_status bdu_update(bdu_handle h, const double *B, const double *C, int64_t r) {
  // transposed form: A^T + C B^T
  if (h && h->tr) return update_common(h, C, B, r, true);
  return update_common(h, B, C, r, true);
}

bdu_status bdu_update_dev(bdu_handle h, const double *dB, const double *dC, int64_t r) {
  if (h && h->tr) return update_common(h, dC, dB, r, false);
  return update_common(h, dB, dC, r, false);
}

// ---------------------------------------------------------------- BHU
// Sec. 3.3, Algorithm 1: the reflectors come from k_bhu.cu; the factors are
// updated as Q <- Q Q_k = Q - (Q Y) SL Y^T and P <- P - (P W) SR W^T.

bdu_status bdu_bhu_sizes(int64_t m, int64_t n, int64_t steps, int64_t *kl, int64_t *kr, int64_t *workspace_bytes) {
  if (m < n || n < 1 || steps < 0 || steps > n || m > (int64_t)1 << 30)
    return fail(nullptr, BDU_EINVAL, "bdu_bhu_sizes: need m >= n >= 1 and 0 <= steps <= n");
  const BhuSizes z = bhu_sizes(m, n, steps);
  if (kl) *kl = z.kl;
  if (kr) *kr = z.kr;
  if (workspace_bytes)
    *workspace_bytes = (int64_t)(sizeof(double) * z.ws_doubles + sizeof(unsigned) * z.ws_counters + sizeof(int) + 16);
  return BDU_OK;
}

bdu_status bdu_bhu_factor(int64_t m, int64_t n, int64_t r, int64_t steps, const double *d, const double *e,
                          const double *u, const double *v, double *alpha, double *beta, double *Y, double *W,
                          double *SL, double *SR, void *workspace, void *stream) {
  if (m < n || n < 1 || steps < 0 || steps > n || m > (int64_t)1 << 30)
    return fail(nullptr, BDU_EINVAL, "bdu_bhu_factor: need m >= n >= 1 and 0 <= steps <= n");
  if (r < 1 || r > BDU_BHU_MAX_RANK) return fail(nullptr, BDU_EINVAL, "bdu_bhu_factor: need 1 <= r <= %d", BDU_BHU_MAX_RANK);
  if (steps == 0) return BDU_OK;
  const BhuSizes z = bhu_sizes(m, n, steps);
  if (!d || !u || !v || !alpha || !workspace || (n > 1 && !e) || (steps > 0 && n > 1 && !beta) ||
      (z.kl > 0 && (!Y || !SL)) || (z.kr > 0 && (!W || !SR)))
    return fail(nullptr, BDU_EINVAL, "bdu_bhu_factor: NULL argument");
  if (((uintptr_t)workspace & 15) != 0) return fail(nullptr, BDU_EINVAL, "bdu_bhu_factor: workspace not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  double *ws = (double *)workspace;
  unsigned *cnt = (unsigned *)(ws + z.ws_doubles);
  int *status = (int *)(cnt + z.ws_counters);
  cudaError_t ce = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * z.ws_counters + sizeof(int), s);
  if (ce == cudaSuccess)
    ce = launch_bhu((int)m, (int)n, (int)steps, (int)r, d, n > 1 ? e : d, u, m, v, n, alpha, n > 1 ? beta : alpha,
                    Y, W, SL, SR, ws, cnt, status, s, nullptr);
  int hst = 0;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return fail(nullptr, BDU_ECUDA, "bdu_bhu_factor: %s", cudaGetErrorString(ce));
  if (hst & ERR_BHU) return fail(nullptr, BDU_ETIMEOUT, "bdu_bhu_factor: a grid barrier ran out");
  return BDU_OK;
}

// ---- the symmetric variant (Sec. 6): A = Q T Q^T, A + rho c c^T

bdu_status bdu_tri_sizes(int64_t n, int64_t steps, int64_t *k, int64_t *workspace_bytes, int64_t *update_bytes) {
  if (n < 1 || steps < 0 || steps > n || n > (int64_t)1 << 30)
    return fail(nullptr, BDU_EINVAL, "bdu_tri_sizes: need n >= 1 and 0 <= steps <= n");
  const BhuSizes z = bhu_sizes(n, n, steps);
  const int64_t ws = (int64_t)(sizeof(double) * z.ws_doubles + sizeof(unsigned) * z.ws_counters + sizeof(int) + 16);
  if (k) *k = z.kr;
  if (workspace_bytes) *workspace_bytes = ws;
  if (update_bytes) {
    const BhuSizes f = bhu_sizes(n, n, n);
    const int64_t kk = f.kr > 0 ? f.kr : 1;
    // the factor's workspace, then u, alpha, beta, Y, S and two n x k products
    const int64_t wsf = (int64_t)(sizeof(double) * f.ws_doubles + sizeof(unsigned) * f.ws_counters + sizeof(int) + 16);
    *update_bytes = ((wsf + 15) / 16) * 16 + (int64_t)sizeof(double) * (3 * (n + 2) + n * kk + kk * kk + 2 * n * kk) + 64;
  }
  return BDU_OK;
}

bdu_status bdu_tri_factor(int64_t n, int64_t steps, const double *a, const double *b, double rho, const double *u,
                          double *alpha, double *beta, double *Y, double *S, void *workspace, void *stream) {
  if (n < 1 || steps < 0 || steps > n || n > (int64_t)1 << 30)
    return fail(nullptr, BDU_EINVAL, "bdu_tri_factor: need n >= 1 and 0 <= steps <= n");
  if (steps == 0) return BDU_OK;
  if (!std::isfinite(rho)) return fail(nullptr, BDU_EINVAL, "bdu_tri_factor: non-finite rho");
  const BhuSizes z = bhu_sizes(n, n, steps);
  if (!a || !u || !alpha || !workspace || (n > 1 && (!b || !beta)) || (z.kr > 0 && (!Y || !S)))
    return fail(nullptr, BDU_EINVAL, "bdu_tri_factor: NULL argument");
  if (((uintptr_t)workspace & 15) != 0) return fail(nullptr, BDU_EINVAL, "bdu_tri_factor: workspace not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  double *ws = (double *)workspace;
  unsigned *cnt = (unsigned *)(ws + z.ws_doubles);
  int *status = (int *)(cnt + z.ws_counters);
  cudaError_t ce = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * z.ws_counters + sizeof(int), s);
  if (ce == cudaSuccess)
    ce = launch_tri((int)n, (int)steps, a, n > 1 ? b : a, rho, u, alpha, n > 1 ? beta : alpha, Y, S, ws, cnt, status, s);
  int hst = 0;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return fail(nullptr, BDU_ECUDA, "bdu_tri_factor: %s", cudaGetErrorString(ce));
  if (hst & ERR_BHU) return fail(nullptr, BDU_ETIMEOUT, "bdu_tri_factor: a grid barrier ran out");
  return BDU_OK;
}

bdu_status bdu_tri_update_dev(int64_t n, double *Q, double *a, double *b, double rho, const double *c,
                              void *workspace, void *stream) {
  if (n < 1 || n > (int64_t)1 << 30) return fail(nullptr, BDU_EINVAL, "bdu_tri_update_dev: need n >= 1");
  if (!Q || !a || !c || !workspace || (n > 1 && !b)) return fail(nullptr, BDU_EINVAL, "bdu_tri_update_dev: NULL argument");
  if (((uintptr_t)workspace & 15) != 0) return fail(nullptr, BDU_EINVAL, "bdu_tri_update_dev: workspace not 16-byte aligned");
  const BhuSizes f = bhu_sizes(n, n, n);
  const int64_t k = f.kr, kk = k > 0 ? k : 1;
  const int64_t wsf = (int64_t)(sizeof(double) * f.ws_doubles + sizeof(unsigned) * f.ws_counters + sizeof(int) + 16);
  char *base = (char *)workspace;
  double *dv = (double *)(base + ((wsf + 15) / 16) * 16);
  double *u = dv, *al = u + (n + 2), *be = al + (n + 2), *Y = be + (n + 2), *S = Y + n * kk, *G1 = S + kk * kk,
         *G2 = G1 + n * kk;
  cudaStream_t s = (cudaStream_t)stream;
  cublasHandle_t cb = nullptr;
  if (cublasCreate(&cb) != CUBLAS_STATUS_SUCCESS) return fail(nullptr, BDU_ENOMEM, "bdu_tri_update_dev: cublasCreate failed");
  bdu_status st = BDU_OK;
  const double one = 1.0, zero = 0.0, minus = -1.0;
  // u = Q^T c
  if (cublasSetStream(cb, s) != CUBLAS_STATUS_SUCCESS ||
      cublasDgemv(cb, CUBLAS_OP_T, (int)n, (int)n, &one, Q, (int)n, c, 1, &zero, u, 1) != CUBLAS_STATUS_SUCCESS)
    st = fail(nullptr, BDU_ECUDA, "bdu_tri_update_dev: the projection failed");
  if (st == BDU_OK) st = bdu_tri_factor(n, n, a, b, rho, u, al, be, Y, S, workspace, stream);
  // Q <- Q - (Q Y) (S Y^T); a, b <- alpha, beta
  if (st == BDU_OK && k > 0 &&
      (cublasDgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)n, (int)k, (int)n, &one, Q, (int)n, Y, (int)n, &zero, G1, (int)n) !=
           CUBLAS_STATUS_SUCCESS ||
       cublasDtrmm(cb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, (int)n, (int)k, &one,
                   S, (int)k, G1, (int)n, G2, (int)n) != CUBLAS_STATUS_SUCCESS ||
       cublasDgemm(cb, CUBLAS_OP_N, CUBLAS_OP_T, (int)n, (int)n, (int)k, &minus, G2, (int)n, Y, (int)n, &one, Q, (int)n) !=
           CUBLAS_STATUS_SUCCESS))
    st = fail(nullptr, BDU_ECUDA, "bdu_tri_update_dev: a cuBLAS product failed");
  if (st == BDU_OK) {
    cudaError_t ce = cudaMemcpyAsync(a, al, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess && n > 1) ce = cudaMemcpyAsync(b, be, sizeof(double) * (n - 1), cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) st = fail(nullptr, BDU_ECUDA, "bdu_tri_update_dev: %s", cudaGetErrorString(ce));
  }
  cublasDestroy(cb);
  return st;
}

static bdu_status bhu_ensure(bdu_ctx *h) {
  if (h->bhu_ws) return BDU_OK;
  const int64_t m = h->m, n = h->n;
  const BhuSizes z = bhu_sizes(m, n, n);
  const int64_t kl = z.kl > 0 ? z.kl : 1, kr = z.kr > 0 ? z.kr : 1;
  h->bhu_Y = (double *)dev_alloc(h, sizeof(double) * m * kl);
  h->bhu_W = (double *)dev_alloc(h, sizeof(double) * n * kr);
  h->bhu_SL = (double *)dev_alloc(h, sizeof(double) * kl * kl);
  h->bhu_SR = (double *)dev_alloc(h, sizeof(double) * kr * kr);
  h->bhu_G1 = (double *)dev_alloc(h, sizeof(double) * m * kl);
  h->bhu_G2 = (double *)dev_alloc(h, sizeof(double) * m * kl);
  h->bhu_vec = (double *)dev_alloc(h, sizeof(double) * 4 * (n + 1));
  h->bhu_cnt = (unsigned *)dev_alloc(h, sizeof(unsigned) * z.ws_counters);
  h->bhu_ws = (double *)dev_alloc(h, sizeof(double) * z.ws_doubles);
  if (!h->bhu_Y || !h->bhu_W || !h->bhu_SL || !h->bhu_SR || !h->bhu_G1 || !h->bhu_G2 || !h->bhu_vec ||
      !h->bhu_cnt || !h->bhu_ws) {
    for (double *p : {h->bhu_Y, h->bhu_W, h->bhu_SL, h->bhu_SR, h->bhu_G1, h->bhu_G2, h->bhu_vec, h->bhu_ws})
      dev_free(h, p);
    dev_free(h, h->bhu_cnt);
    h->bhu_Y = h->bhu_W = h->bhu_SL = h->bhu_SR = h->bhu_G1 = h->bhu_G2 = h->bhu_vec = h->bhu_ws = nullptr;
    h->bhu_cnt = nullptr;
    return fail(h, BDU_ENOMEM, "device allocation for the BHU workspace failed");
  }
  cudaError_t ce = cudaMemsetAsync(h->bhu_cnt, 0, sizeof(unsigned) * z.ws_counters, h->stream);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "clearing the BHU counters");
  if (!h->cublas) {
    cublasHandle_t cb = nullptr;
    if (cublasCreate(&cb) != CUBLAS_STATUS_SUCCESS) return fail(h, BDU_ENOMEM, "cublasCreate failed");
    h->cublas = cb;
  }
  return BDU_OK;
}

// X <- X - (X Yr) S Yr^T for X rows x k reflectors (column-major, ld rows).
static bool bhu_apply_factor(cublasHandle_t cb, double *X, int64_t rows, const double *Yr, int64_t k,
                             const double *S, double *G1, double *G2) {
  const double one = 1.0, zero = 0.0, minus = -1.0;
  if (k <= 0) return true;
  return cublasDgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)rows, (int)k, (int)rows, &one, X, (int)rows, Yr, (int)rows,
                     &zero, G1, (int)rows) == CUBLAS_STATUS_SUCCESS &&
         cublasDtrmm(cb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, (int)rows,
                     (int)k, &one, S, (int)k, G1, (int)rows, G2, (int)rows) == CUBLAS_STATUS_SUCCESS &&
         cublasDgemm(cb, CUBLAS_OP_N, CUBLAS_OP_T, (int)rows, (int)rows, (int)k, &minus, G2, (int)rows, Yr,
                     (int)rows, &one, X, (int)rows) == CUBLAS_STATUS_SUCCESS;
}

static bdu_status run_update_bhu(bdu_ctx *h, const double *dB, const double *dC, int64_t r) {
  bdu_status st = flush_apply(h);
  if (st != BDU_OK) return st;
  st = bhu_ensure(h);
  if (st != BDU_OK) return st;
  const int64_t m = h->m, n = h->n;
  const BhuSizes z = bhu_sizes(m, n, n);
  cudaStream_t s = h->stream;
  cublasHandle_t cb = (cublasHandle_t)h->cublas;
  if (cublasSetStream(cb, s) != CUBLAS_STATUS_SUCCESS) return fail(h, BDU_EINTERNAL, "cublasSetStream failed");
  double *d = h->bhu_vec, *e = d + (n + 1), *alpha = e + (n + 1), *beta = alpha + (n + 1);
  int64_t launches = 0;
  // direct rank-r absorption: up to BDU_BHU_MAX_RANK columns per sweep
  for (int64_t k0 = 0; k0 < r; k0 += BDU_BHU_MAX_RANK) {
    const int rc = (int)std::min<int64_t>(BDU_BHU_MAX_RANK, r - k0);
    // U = Q^T B(:, k0..), V = P^T C(:, k0..) with the current factors
    cudaError_t ce = launch_project_nz(BDU_FP64, h->Q, m, (int)m, (int)m, dB + k0 * m, m, rc, h->U, m, h->nzB, s);
    if (ce == cudaSuccess) ce = launch_project_nz(BDU_FP64, h->P, n, (int)n, (int)n, dC + k0 * n, n, rc, h->V, n, h->nzC, s);
    if (ce == cudaSuccess) ce = launch_bhu_band_get(h->band, (int)m, (int)n, d, e, s);
    if (ce == cudaSuccess)
      ce = launch_bhu((int)m, (int)n, (int)n, rc, d, e, h->U, m, h->V, n, alpha, beta, h->bhu_Y, h->bhu_W, h->bhu_SL,
                      h->bhu_SR, h->bhu_ws, h->bhu_cnt, h->status, s, &launches);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "BHU reflectors");
    if (!bhu_apply_factor(cb, (double *)h->Q, m, h->bhu_Y, z.kl, h->bhu_SL, h->bhu_G1, h->bhu_G2) ||
        !bhu_apply_factor(cb, (double *)h->P, n, h->bhu_W, z.kr, h->bhu_SR, h->bhu_G1, h->bhu_G2))
      return fail(h, BDU_ECUDA, "BHU: a cuBLAS product failed");
    ce = launch_bhu_band_put(h->band, (int)m, (int)n, alpha, beta, s);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "BHU: storing the bidiagonal");
    launches += 6;
    h->updates += rc;
    h->bhu_updates++;
  }
  h->launches += launches;
  return BDU_OK;
}

static bdu_status update_bhu_common(bdu_handle h, const double *B, const double *C, int64_t r, bool host) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (h->poisoned) return fail(h, BDU_EPOISONED, "handle poisoned by an earlier failure: %s", h->err);
  if (h->opt.precision != BDU_FP64) return fail(h, BDU_EINVAL, "BHU updates need an FP64 handle");
  if (r < 0) return fail(h, BDU_EINVAL, "negative rank %lld", (long long)r);
  if (r == 0) return BDU_OK;
  if (!B || !C) return fail(h, BDU_EINVAL, "NULL update pointer");
  if (r > 4096) return fail(h, BDU_EINVAL, "rank %lld exceeds 4096", (long long)r);
  if (host && (!all_finite(B, h->m * r) || !all_finite(C, h->n * r)))
    return fail(h, BDU_EINVAL, "non-finite value in B or C");
  cudaError_t ce = cudaSetDevice(h->device);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaSetDevice");
  bdu_status st = ensure_rank_workspace(h, r);
  if (st != BDU_OK) return st;
  const double *dB = B, *dC = C;
  if (host) {
    ce = cudaMemcpyAsync(h->dB, B, sizeof(double) * h->m * r, cudaMemcpyHostToDevice, h->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h->dC, C, sizeof(double) * h->n * r, cudaMemcpyHostToDevice, h->stream);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "copying B, C to the device");
    dB = h->dB; dC = h->dC;
  }
  return run_update_bhu(h, dB, dC, r);
}

bdu_status bdu_update_bhu(bdu_handle h, const double *B, const double *C, int64_t r) {
  if (h && h->tr) return update_bhu_common(h, C, B, r, true);
  return update_bhu_common(h, B, C, r, true);
}

bdu_status bdu_update_bhu_dev(bdu_handle h, const double *dB, const double *dC, int64_t r) {
  if (h && h->tr) return update_bhu_common(h, dC, dB, r, false);
  return update_bhu_common(h, dB, dC, r, false);
}

static bdu_status update_batch_held(bdu_handle *hs, int count, const double *const *dB, const double *const *dC,
                                    const int64_t *r, void *stream);

bdu_status bdu_update_batch(bdu_handle *hs, int count, const double *const *dB, const double *const *dC,
                            const int64_t *r, void *stream) {
  if (count <= 0 || !hs || !dB || !dC) return update_batch_held(hs, count, dB, dC, r, stream);
  // B and C trade places for the handles held in transposed form
  std::vector<const double *> b(dB, dB + count), c(dC, dC + count);
  for (int i = 0; i < count; i++)
    if (hs[i] && hs[i]->tr) std::swap(b[i], c[i]);
  return update_batch_held(hs, count, b.data(), c.data(), r, stream);
}

static bdu_status update_batch_held(bdu_handle *hs, int count, const double *const *dB, const double *const *dC,
                                    const int64_t *r, void *stream) {
  if (count < 0) return fail(nullptr, BDU_EINVAL, "bdu_update_batch: negative count");
  if (count == 0) return BDU_OK;
  if (!hs || !dB || !dC || !r) return fail(nullptr, BDU_EINVAL, "bdu_update_batch: NULL argument");
  for (int i = 0; i < count; i++) {
    if (!hs[i]) return fail(nullptr, BDU_EINVAL, "bdu_update_batch: NULL handle at %d", i);
    if (r[i] < 0 || r[i] > 4096) return fail(hs[i], BDU_EINVAL, "bdu_update_batch: bad rank %lld", (long long)r[i]);
    if (r[i] > 0 && (!dB[i] || !dC[i])) return fail(hs[i], BDU_EINVAL, "bdu_update_batch: NULL update pointer");
    if (hs[i]->opt.precision != hs[0]->opt.precision || hs[i]->device != hs[0]->device)
      return fail(hs[i], BDU_EINVAL, "bdu_update_batch: handles differ in precision or device");
    for (int j = 0; j < i; j++)
      if (hs[j] == hs[i]) return fail(hs[i], BDU_EINVAL, "bdu_update_batch: handle %d repeated", i);
  }
  BatchGuard bg;
  for (int i = 0; i < count; i++) {
    int expect = 0;
    if (!hs[i]->busy.compare_exchange_strong(expect, 1)) return fail(hs[i], BDU_EBUSY, "handle in use by another thread");
    bg.held.push_back(hs[i]);
    if (hs[i]->poisoned) return fail(hs[i], BDU_EPOISONED, "handle poisoned by an earlier failure");
  }
  bdu_ctx *h0 = hs[0];
  const int precision = h0->opt.precision;
  cudaError_t ce = cudaSetDevice(h0->device);
  if (ce != cudaSuccess) return cuda_fail(h0, ce, "cudaSetDevice");
  for (int i = 0; i < count; i++) {
    bdu_status fs = flush_apply(hs[i]);
    if (fs != BDU_OK) return fs;
  }
  cudaStream_t s = stream ? (cudaStream_t)stream : h0->stream;
  int64_t max_r = 0;
  for (int i = 0; i < count; i++) {
    bdu_status st = ensure_rank_workspace(hs[i], r[i] > 0 ? r[i] : 1);
    if (st != BDU_OK) return st;
    if (r[i] > max_r) max_r = r[i];
  }
  // order the batch after each handle's pending work
  for (int i = 0; i < count; i++)
    if (hs[i]->stream != s) {
      cudaEvent_t ev;
      ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = cudaEventRecord(ev, hs[i]->stream);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ev, 0);
      cudaEventDestroy(ev);
      if (ce != cudaSuccess) return cuda_fail(hs[i], ce, "ordering a batch");
    }
  // descriptor workspace
  const size_t need = sizeof(ChaseArgs) * count + sizeof(ApplyItem) * 2 * count + sizeof(ProjItem) * 2 * count +
                      sizeof(int) * (2 * count + 2) + sizeof(double *) * 2 * count + 1024;
  if (h0->batch_ws_bytes < need) {
    void *p = dev_alloc(h0, need);
    if (!p) return fail(h0, BDU_ENOMEM, "batch descriptor allocation failed");
    dev_free(h0, h0->batch_ws);
    h0->batch_ws = p;
    h0->batch_ws_bytes = need;
  }
  char *ws = (char *)h0->batch_ws;
  ChaseArgs *d_chase = (ChaseArgs *)ws;
  ApplyItem *d_apply = (ApplyItem *)(ws + sizeof(ChaseArgs) * count);
  ProjItem *d_proj = (ProjItem *)((char *)d_apply + sizeof(ApplyItem) * 2 * count);
  int *d_first = (int *)((char *)d_proj + sizeof(ProjItem) * 2 * count);
  const double **d_cols = (const double **)(((uintptr_t)(d_first + 2 * count + 2) + 15) & ~(uintptr_t)15);

  // K1: projections of all items, one launch
  std::vector<ProjItem> proj;
  int max_nrow = 0;
  for (int i = 0; i < count; i++) {
    if (r[i] == 0) continue;
    bdu_ctx *h = hs[i];
    proj.push_back({h->Q, (int)h->m, (int)h->m, (int)r[i], dB[i], h->U, h->nzB});
    proj.push_back({h->P, (int)h->n, (int)h->n, (int)r[i], dC[i], h->V, h->nzC});
    if (h->m > max_nrow) max_nrow = (int)h->m;
  }
  if (proj.empty()) return BDU_OK;
  ce = cudaMemcpyAsync(d_proj, proj.data(), sizeof(ProjItem) * proj.size(), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = launch_project_batch(precision, d_proj, (int)proj.size(), max_nrow, max_nrow, (int)max_r, s);
  if (ce != cudaSuccess) return cuda_fail(h0, ce, "batched projection");

  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int esz = precision == BDU_FP64 ? 8 : 4;
  if (!h0->batch_aux && cudaStreamCreateWithFlags(&h0->batch_aux, cudaStreamNonBlocking) != cudaSuccess) {
    h0->batch_aux = nullptr;
    return cuda_fail(h0, cudaGetLastError(), "creating the batch stream");
  }
  for (int64_t k = 0; k < max_r; k++) {
    // small items (one thread block each) first, then large ones (a cluster each)
    std::vector<ChaseArgs> chase_s, chase_l;
    std::vector<const double *> ucol_s, ucol_l, vcol_s, vcol_l;
    std::vector<ApplyItem> apply;
    std::vector<std::pair<bdu_ctx *, int>> tc_items;  // (handle, side) applied by the blocked apply
    std::vector<int> first;
    int max_n = 0, max_n_l = 0, max_band = 0, slabs = 0;
    size_t smem = 0;
    for (int i = 0; i < count; i++) {
      if (r[i] <= k) continue;
      bdu_ctx *h = hs[i];
      const int m = (int)h->m, n = (int)h->n;
      ChaseArgs a{};
      a.m = m; a.n = n; a.band = band_ptrs(h->band, m, n);
      const bool after = precision == BDU_MIXED && rotate_vectors_supported(m, n);
      a.rx = after ? 0 : (int)(r[i] - k - 1);
      a.Ux = a.rx > 0 ? h->U + (k + 1) * m : nullptr;
      a.Vx = a.rx > 0 ? h->V + (k + 1) * n : nullptr;
      a.st = h->st; a.status = h->status; a.counters = h->counters;
      a.fast = precision == BDU_MIXED ? 1 : 0;
      a.step_budget = h->opt.step_budget;
      if (n >= kClusterBatchMinN && chase_cluster_fits(m, n)) {
        a.engine = 2;
        chase_l.push_back(a);
        ucol_l.push_back(h->U + k * m);
        vcol_l.push_back(h->V + k * n);
        if (n > max_n_l) max_n_l = n;
      } else {
        a.engine = 1;
        chase_s.push_back(a);
        ucol_s.push_back(h->U + k * m);
        vcol_s.push_back(h->V + k * n);
        if (n > max_n) max_n = n;
        if ((int)band_doubles(m, n) > max_band) max_band = (int)band_doubles(m, n);
      }
      for (int side = 0; side < 2; side++) {
        const int dim = side == 0 ? m : n;
        if (precision == BDU_MIXED && dim >= kBlockedFrom && h->st.tc_ws) {
          tc_items.push_back({h, side});  // the blocked apply, as a single update takes it
          continue;
        }
        ApplyItem it{};
        it.X = side == 0 ? h->Q : h->P;
        it.ld = side == 0 ? m : n;
        it.nrow = it.ncol = side == 0 ? m : n;
        apply_geometry(precision, it.ncol, (size_t)optin, &it.R, &it.csw);
        if (it.R == 0) return fail(h, BDU_EINVAL, "matrix too wide for the batched apply");
        it.side = side;
        it.with_spike = (side == 0 && m > n) ? 1 : 0;
        it.st = h->st;
        first.push_back(slabs);
        slabs += (it.nrow + it.R - 1) / it.R;
        const size_t sm = (size_t)esz * it.csw * it.ncol;
        if (sm > smem) smem = sm;
        apply.push_back(it);
      }
    }
    const int ns = (int)chase_s.size(), nl = (int)chase_l.size(), nact = ns + nl;
    std::vector<ChaseArgs> chase(chase_s);
    chase.insert(chase.end(), chase_l.begin(), chase_l.end());
    std::vector<const double *> cols(ucol_s);  // u columns then v columns, in chase order
    cols.insert(cols.end(), ucol_l.begin(), ucol_l.end());
    cols.insert(cols.end(), vcol_s.begin(), vcol_s.end());
    cols.insert(cols.end(), vcol_l.begin(), vcol_l.end());
    first.push_back(slabs);
    ce = cudaMemcpyAsync(d_chase, chase.data(), sizeof(ChaseArgs) * nact, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_cols, cols.data(), sizeof(double *) * cols.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_apply, apply.data(), sizeof(ApplyItem) * apply.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = launch_stage_batch(d_chase, d_cols, d_cols + nact, nact, s);
    // the small items' chases on the second stream, beside the large items'
    cudaEvent_t fork = nullptr, join = nullptr;
    if (ce == cudaSuccess && ns > 0 && nl > 0) {
      ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = cudaEventRecord(fork, s);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h0->batch_aux, fork, 0);
    }
    const cudaStream_t ss = (ns > 0 && nl > 0) ? h0->batch_aux : s;
    if (ce == cudaSuccess && ns > 0) ce = launch_chase_batch(d_chase, ns, max_n, max_band, precision == BDU_MIXED, ss);
    if (ce == cudaSuccess && nl > 0)
      ce = launch_chase_cluster_batch(d_chase + ns, nl, max_n_l, precision == BDU_MIXED, s);
    if (ce == cudaSuccess && join) {
      ce = cudaEventRecord(join, h0->batch_aux);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, join, 0);
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    // mixed form: each item's later projections, rotated by this round's rotations
    for (int i = 0; i < count && ce == cudaSuccess; i++) {
      bdu_ctx *h = hs[i];
      const int m = (int)h->m, n = (int)h->n, later = (int)(r[i] - k - 1);
      if (later <= 0 || precision != BDU_MIXED || !rotate_vectors_supported(m, n)) continue;
      ce = launch_chase_descriptors(h->st, 0, s);
      if (ce == cudaSuccess) ce = launch_chase_descriptors(h->st, 1, s);
      if (ce == cudaSuccess)
        ce = launch_rotate_vector_sets(h->U + (k + 1) * m, h->U + (k + 1) * m, m, later, m, h->V + (k + 1) * n,
                                       h->V + (k + 1) * n, n, later, n, h->st, m > n, h->status, s);
      h0->launches += 3;
    }
    if (ce == cudaSuccess) ce = launch_apply_batch(precision, d_apply, d_first, (int)apply.size(), slabs, smem, s);
    for (size_t q = 0; q < tc_items.size() && ce == cudaSuccess; q++) {
      bdu_ctx *h = tc_items[q].first;
      const int side = tc_items[q].second, dim = side == 0 ? (int)h->m : (int)h->n;
      ce = launch_apply_tc((float *)(side == 0 ? h->Q : h->P), dim, dim, dim, h->st, side,
                           side == 0 && h->m > h->n, h->status, false, 128, h->st.tc_ws, h->st.tc_ws_bytes, s);
    }
    if (ce != cudaSuccess) return cuda_fail(h0, ce, "batched update round");
    h0->launches += 3;
    for (int i = 0; i < count; i++)
      if (r[i] > k) {
        const bdu_status rs = reorth_after_column(hs[i], s);
        if (rs != BDU_OK) return rs;
      }
  }
  h0->launches += 2;
  // each handle's later work waits for the batch
  cudaEvent_t done;
  ce = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventRecord(done, s);
  for (int i = 0; i < count && ce == cudaSuccess; i++)
    if (hs[i]->stream != s) ce = cudaStreamWaitEvent(hs[i]->stream, done, 0);
  cudaEventDestroy(done);
  if (ce != cudaSuccess) return cuda_fail(h0, ce, "ordering after a batch");
  for (int i = 0; i < count; i++) {
    hs[i]->updates += r[i];
    bdu_status st = maybe_reorth(hs[i], r[i]);
    if (st != BDU_OK) return st;
  }
  return BDU_OK;
}

bdu_status bdu_sync(bdu_handle h) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (h->poisoned) return fail(h, BDU_EPOISONED, "handle poisoned by an earlier failure");
  cudaSetDevice(h->device);
  bdu_status st = flush_apply(h);
  if (st == BDU_OK) st = settle_probe(h);
  return st != BDU_OK ? st : check_device_status(h);
}

bdu_status bdu_flush(bdu_handle h) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (h->poisoned) return fail(h, BDU_EPOISONED, "handle poisoned by an earlier failure");
  cudaSetDevice(h->device);
  return flush_apply(h);
}

bdu_status bdu_read(bdu_handle h, double *Q, double *d, double *e, double *P) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  if (h->tr) std::swap(Q, P);
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  cudaSetDevice(h->device);
  bdu_status st = BDU_OK;
  if (!h->poisoned && (Q || P)) st = flush_apply(h);  // d and e are current without it
  if (st == BDU_OK && !h->poisoned) st = settle_probe(h);
  if (st == BDU_OK && !h->poisoned) st = check_device_status(h);
  const int64_t m = h->m, n = h->n;
  cudaError_t ce = cudaSuccess;
  auto fetch = [&](void *src, double *dst, int64_t count) {
    if (!dst || ce != cudaSuccess) return;
    if (h->opt.precision == BDU_FP64) {
      ce = cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream);
    } else {
      ce = launch_convert_f32_to_f64((const float *)src, h->scratch64, count, h->stream);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(dst, h->scratch64, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    }
  };
  fetch(h->Q, Q, m * m);
  fetch(h->P, P, n * n);
  if ((d || e) && ce == cudaSuccess) ce = read_bidiagonal(h, d, e);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_read");
  return st;
}

bdu_status bdu_read_rotations(bdu_handle h, int side, double *c, double *s, int32_t *a,
                              int64_t cap, int64_t *count) {
  if (!h || !count || (side != 0 && side != 1)) return fail(h, BDU_EINVAL, "bdu_read_rotations: bad argument");
  if (h->tr) side ^= 1;  // the rotations on the caller's Q act on the held P
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  cudaSetDevice(h->device);
  cudaError_t ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_read_rotations");
  const RotStream &st = h->st;
  const size_t tc = (size_t)st.T * st.cap;
  std::vector<int32_t> cnt(st.T + 1, 0);
  std::vector<double> hc(tc), hs(tc);
  std::vector<int32_t> ha(tc);
  ce = cudaMemcpy(cnt.data(), side == 0 ? st.Ln : st.Rn, sizeof(int32_t) * st.T, cudaMemcpyDeviceToHost);
  const double *dc = side == 0 ? st.Lc : st.Rc;
  if (dc) {
    if (ce == cudaSuccess) ce = cudaMemcpy(hc.data(), dc, sizeof(double) * tc, cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(hs.data(), side == 0 ? st.Ls : st.Rs, sizeof(double) * tc, cudaMemcpyDeviceToHost);
  } else {
    // mixed form: the FP32 coefficients the factors are rotated with
    std::vector<float2> hf(tc);
    if (ce == cudaSuccess) ce = cudaMemcpy(hf.data(), side == 0 ? st.Lf : st.Rf, sizeof(float2) * tc, cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < tc; i++) { hc[i] = hf[i].x; hs[i] = hf[i].y; }
  }
  if (ce == cudaSuccess) ce = cudaMemcpy(ha.data(), side == 0 ? st.La : st.Ra, sizeof(int32_t) * tc, cudaMemcpyDeviceToHost);
  int32_t ns = 0;
  std::vector<double> sc, ss;
  std::vector<int32_t> sa;
  if (ce == cudaSuccess && side == 0 && h->m > h->n) {
    ce = cudaMemcpy(&ns, st.Sn, sizeof(int32_t), cudaMemcpyDeviceToHost);
    sc.resize(ns + 1); ss.resize(ns + 1); sa.resize(ns + 1);
    if (dc) {
      if (ce == cudaSuccess && ns > 0) ce = cudaMemcpy(sc.data(), st.Sc, sizeof(double) * ns, cudaMemcpyDeviceToHost);
      if (ce == cudaSuccess && ns > 0) ce = cudaMemcpy(ss.data(), st.Ss, sizeof(double) * ns, cudaMemcpyDeviceToHost);
    } else {
      std::vector<float2> sf(ns + 1);
      if (ce == cudaSuccess && ns > 0) ce = cudaMemcpy(sf.data(), st.Sf, sizeof(float2) * ns, cudaMemcpyDeviceToHost);
      for (int32_t q = 0; q < ns; q++) { sc[q] = sf[q].x; ss[q] = sf[q].y; }
    }
    if (ce == cudaSuccess && ns > 0) ce = cudaMemcpy(sa.data(), st.Sa, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost);
  }
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_read_rotations");
  int64_t k = 0;
  auto put = [&](double cc, double sv, int32_t aa) {
    if (k < cap) {
      if (c) c[k] = cc;
      if (s) s[k] = sv;
      if (a) a[k] = aa;
    }
    k++;
  };
  for (int32_t q = 0; q < ns; q++) put(sc[q], ss[q], sa[q]);
  for (int t = 0; t < st.T; t++)
    for (int32_t q = 0; q < cnt[t] && q < st.cap; q++) {
      const size_t i = (size_t)t * st.cap + q;
      put(hc[i], hs[i], ha[i]);
    }
  *count = k;
  return BDU_OK;
}

bdu_status bdu_read_truncated(bdu_handle h, int64_t r, double *L, double *R, int64_t *idx, double *err2) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  if (h->tr) std::swap(L, R);  // A_r = (L' R'^T)^T for the held A^T
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (r < 0 || r > h->n) return fail(h, BDU_EINVAL, "bdu_read_truncated: need 0 <= r <= min(m, n) (r=%lld)", (long long)r);
  cudaSetDevice(h->device);
  bdu_status st = BDU_OK;
  if (!h->poisoned) st = flush_apply(h);
  if (st == BDU_OK && !h->poisoned) st = settle_probe(h);
  if (st == BDU_OK && !h->poisoned) st = check_device_status(h);
  if (st != BDU_OK) return st;
  const int64_t m = h->m, n = h->n;
  std::vector<double> d(n), e(n > 1 ? n - 1 : 1);
  cudaError_t ce = read_bidiagonal(h, d.data(), e.data());
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_read_truncated");
  // weights alpha_i^2 + beta_{i-1}^2 (Eq. errtrBD), each product rounded on its
  // own (volatile keeps the host compiler from fusing them into an FMA); the r
  // largest, lower i first on ties
  std::vector<double> w(n);
  for (int64_t i = 0; i < n; i++) {
    volatile double a2 = d[i] * d[i];
    if (i == 0) {
      w[i] = a2;
    } else {
      volatile double b2 = e[i - 1] * e[i - 1];
      w[i] = a2 + b2;
    }
  }
  std::vector<int64_t> order(n);
  for (int64_t i = 0; i < n; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return w[a] > w[b]; });
  std::vector<int64_t> keep(order.begin(), order.begin() + r);
  std::sort(keep.begin(), keep.end());
  std::vector<char> kept(n, 0);
  for (int64_t i : keep) kept[i] = 1;
  double err = 0.0;
  for (int64_t i = 0; i < n; i++)
    if (!kept[i]) err = err + w[i];
  if (err2) *err2 = err;
  if (idx)
    for (int64_t k = 0; k < r; k++) idx[k] = keep[k] + 1;
  if (r == 0 || (!L && !R)) return BDU_OK;
  // the columns of L and R, formed on the device
  std::vector<int32_t> hi(r);
  std::vector<double> ha(r), hbt(r);
  for (int64_t k = 0; k < r; k++) {
    const int64_t i = keep[k];
    hi[k] = (int32_t)(i + 1);
    ha[k] = d[i];
    hbt[k] = i > 0 ? e[i - 1] : 0.0;
  }
  const size_t bytes = sizeof(double) * (size_t)(m + n) * r + sizeof(double) * 2 * r + sizeof(int32_t) * r + 64;
  char *ws = (char *)dev_alloc(h, bytes);
  if (!ws) return fail(h, BDU_ENOMEM, "bdu_read_truncated: workspace allocation failed");
  double *dL = (double *)ws;
  double *dR = dL + (size_t)m * r;
  double *da = dR + (size_t)n * r;
  double *db = da + r;
  int32_t *di = (int32_t *)(db + r);
  cudaStream_t s = h->stream;
  ce = cudaMemcpyAsync(da, ha.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(db, hbt.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(di, hi.data(), sizeof(int32_t) * r, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = launch_truncate(h->opt.precision, h->Q, m, h->P, n, di, da, db, (int)r, dL, dR, s);
  if (ce == cudaSuccess && L) ce = cudaMemcpyAsync(L, dL, sizeof(double) * (size_t)m * r, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess && R) ce = cudaMemcpyAsync(R, dR, sizeof(double) * (size_t)n * r, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  dev_free(h, ws);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_read_truncated");
  h->launches += 1;
  return BDU_OK;
}

bdu_status bdu_singular_values(bdu_handle h, int64_t k, double *sv) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (k < 0 || k > h->n) return fail(h, BDU_EINVAL, "bdu_singular_values: need 0 <= k <= min(m, n) (k=%lld)", (long long)k);
  if (k > 0 && !sv) return fail(h, BDU_EINVAL, "bdu_singular_values: NULL output");
  cudaSetDevice(h->device);
  bdu_status st = BDU_OK;
  if (!h->poisoned) st = settle_probe(h);
  if (st == BDU_OK && !h->poisoned) st = check_device_status(h);
  if (st != BDU_OK) return st;
  if (k == 0) return BDU_OK;
  const int64_t n = h->n;
  std::vector<double> d(n), e(n > 1 ? n - 1 : 1);
  cudaError_t ce = read_bidiagonal(h, d.data(), e.data());
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_singular_values");
  // Golub-Kahan off-diagonal d_1, e_1, ..., d_n: squares, a Gershgorin bound
  // of sigma_max and the smallest pivot magnitude
  std::vector<double> b2(2 * n - 1);
  double bmax2 = 0.0, hi = 0.0, prev = 0.0;
  for (int64_t i = 0; i < 2 * n - 1; i++) {
    const double b = fabs((i & 1) ? e[i / 2] : d[i / 2]);
    b2[i] = b * b;
    bmax2 = b2[i] > bmax2 ? b2[i] : bmax2;
    hi = prev + b > hi ? prev + b : hi;
    prev = b;
  }
  hi = prev > hi ? prev : hi;
  hi = hi * (1.0 + 8.0 * DBL_EPSILON) + DBL_MIN;
  const double pivmin = DBL_MIN * (bmax2 > 1.0 ? bmax2 : 1.0);
  const size_t bytes = sizeof(double) * (size_t)(2 * n - 1 + k) + 64;
  double *ws = (double *)dev_alloc(h, bytes);
  if (!ws) return fail(h, BDU_ENOMEM, "bdu_singular_values: workspace allocation failed");
  double *db2 = ws, *dsv = ws + (2 * n - 1);
  cudaStream_t s = h->stream;
  ce = cudaMemcpyAsync(db2, b2.data(), sizeof(double) * b2.size(), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = launch_bidiag_svals(db2, (int)n, hi, pivmin, (int)k, dsv, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(sv, dsv, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  dev_free(h, ws);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_singular_values");
  h->launches += 1;
  return BDU_OK;
}

bdu_status bdu_stats(bdu_handle h, bdu_stats_t *out) {
  if (!h || !out) return fail(h, BDU_EINVAL, "bdu_stats: bad argument");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  cudaSetDevice(h->device);
  if (!h->poisoned) {
    bdu_status sp = settle_probe(h);
    if (sp != BDU_OK) return sp;
  }
  unsigned long long c[16];
  cudaError_t ce = cudaMemcpyAsync(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_stats");
  memset(out, 0, sizeof(*out));
  out->updates = h->updates;
  for (int q = 0; q < 4; q++) {
    out->rot_left[q] = (int64_t)c[q];
    out->rot_right[q] = (int64_t)c[4 + q];
  }
  out->chase_steps = (int64_t)c[8];
  out->ortho_q = h->ortho[0];
  out->ortho_p = h->ortho[1];
  out->reorth_q = h->reorth[0];
  out->reorth_p = h->reorth[1];
  resolve_timers(h);
  out->launches = h->launches;
  out->timed_updates = h->timed_updates;
  out->ms_project = h->ms[0];
  out->ms_chase = h->ms[1];
  out->ms_apply_q = h->ms[2];
  out->ms_apply_p = h->ms[3];
  out->apply_launches = h->apply_launches;
  int64_t bytes = 0;
  for (size_t b : h->block_bytes) bytes += (int64_t)b;
  out->device_bytes = bytes;
  out->graph_replays = h->graph_replays;
  out->apply_variant[0] = h->apply_var[0];
  out->apply_variant[1] = h->apply_var[1];
  out->tunings = h->tunings;
  if (h->tr) {
    // left = on the caller's Q, which is the held P
    for (int q = 0; q < 4; q++) std::swap(out->rot_left[q], out->rot_right[q]);
    std::swap(out->ortho_q, out->ortho_p);
    std::swap(out->reorth_q, out->reorth_p);
    std::swap(out->ms_apply_q, out->ms_apply_p);
    std::swap(out->apply_variant[0], out->apply_variant[1]);
  }
  return BDU_OK;
}

bdu_status bdu_check_orthogonality(bdu_handle h, double *q_est, double *p_est) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (h->poisoned) return fail(h, BDU_EPOISONED, "handle poisoned by an earlier failure");
  cudaSetDevice(h->device);
  double e0 = 0.0, e1 = 0.0;
  bdu_status st = settle_probe(h);
  if (st == BDU_OK) st = probe_factor(h, 0, &e0);
  if (st == BDU_OK) st = probe_factor(h, 1, &e1);
  if (st != BDU_OK) return st;
  if (h->tr) std::swap(e0, e1);
  if (q_est) *q_est = e0;
  if (p_est) *p_est = e1;
  return BDU_OK;
}

bdu_status bdu_set_fault_injection(int site, int64_t value) {
  if (site == BDU_INJECT_NONE) {
    g_inject_site.store(BDU_INJECT_NONE);
    g_inject_value.store(0);
    return BDU_OK;
  }
  if (site < BDU_INJECT_STEP_BUDGET || site > BDU_INJECT_BHU_STALL || value < 1) return BDU_EINVAL;
  g_inject_value.store(value);
  g_inject_site.store(site);
  return BDU_OK;
}

bdu_status bdu_set_timing(bdu_handle h, int on) {
  if (!h) return fail(nullptr, BDU_EINVAL, "NULL handle");
  Guard g(h);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  cudaSetDevice(h->device);
  h->timing = on != 0;
  return BDU_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Rank-k tracking (Sec. 4, Eqs. lrup, defup, qrlr, equivlrup, bdlrup).  The
// thin factors [Q1, new column] and [P1, new column] live in device buffers of
// k+1 columns (FP64, or FP32 in the mixed form); the (k+1)-order middle matrix
// is reduced by an internal handle of the same form (the chase and application
// kernels of the full update) whose factors are reset to the identity before
// every step, so that afterwards they hold Q2 and P2.  The projections
// (classical Gram-Schmidt, twice) and the products [Q1, q] Q2(:, kept) are
// cuBLAS BLAS-2/3 calls: the products are plain GEMMs, the step's largest cost
// for m, n >> k.  The mixed form follows each step with one Newton-Schulz step
// on Q1 and P1 (as the full mixed form does for Q and P).
// ---------------------------------------------------------------------------
struct bdu_thin_ctx {
  int64_t m, n, k;
  bool mixed = false;
  bdu_ctx *core = nullptr;
  void *Qb = nullptr, *Pb = nullptr, *Qn = nullptr, *Pn = nullptr;  // m x (k+1), n x (k+1)
  void *x = nullptr, *y = nullptr, *r = nullptr, *zq = nullptr, *zp = nullptr;
  void *h1 = nullptr, *h2 = nullptr, *wq = nullptr, *wp = nullptr, *ones = nullptr, *K2 = nullptr;
  double *u = nullptr, *v = nullptr, *xd = nullptr;  // FP64 middle-matrix vectors; FP64 staging (mixed)
  float *E = nullptr, *W = nullptr;                  // re-orthogonalization workspace (mixed)
  std::vector<double> d, e;
  double delta_host[2] = {0.0, 0.0};
  int64_t updates = 0, in_span_b = 0, in_span_c = 0;
  std::atomic<int> busy{0};
};

namespace {

constexpr double kThinTau64 = 0x1p-40;                // b in span(Q1) when ||b_perp|| <= tau ||b||
constexpr double kThinTau32 = 0x1p-16;                // the same for FP32 factors
constexpr double kGolden = 0.6180339887498949;        // FP64 nearest (sqrt(5) - 1) / 2

struct ThinGuard {
  bdu_thin_ctx *t;
  bool ok;
  explicit ThinGuard(bdu_thin_ctx *tt) : t(tt), ok(false) {
    int expect = 0;
    ok = t->busy.compare_exchange_strong(expect, 1);
  }
  ~ThinGuard() {
    if (ok) t->busy.store(0);
  }
};

// cuBLAS by element type
inline cublasStatus_t bl_gemv(cublasHandle_t h, cublasOperation_t op, int m, int n, const double *a,
                              const double *A, int lda, const double *x, const double *b, double *y) {
  return cublasDgemv(h, op, m, n, a, A, lda, x, 1, b, y, 1);
}
inline cublasStatus_t bl_gemv(cublasHandle_t h, cublasOperation_t op, int m, int n, const float *a, const float *A,
                              int lda, const float *x, const float *b, float *y) {
  return cublasSgemv(h, op, m, n, a, A, lda, x, 1, b, y, 1);
}
inline cublasStatus_t bl_copy(cublasHandle_t h, int n, const double *x, int incx, double *y, int incy) {
  return cublasDcopy(h, n, x, incx, y, incy);
}
inline cublasStatus_t bl_copy(cublasHandle_t h, int n, const float *x, int incx, float *y, int incy) {
  return cublasScopy(h, n, x, incx, y, incy);
}
inline cublasStatus_t bl_axpy(cublasHandle_t h, int n, const double *a, const double *x, double *y) {
  return cublasDaxpy(h, n, a, x, 1, y, 1);
}
inline cublasStatus_t bl_axpy(cublasHandle_t h, int n, const float *a, const float *x, float *y) {
  return cublasSaxpy(h, n, a, x, 1, y, 1);
}
inline cublasStatus_t bl_nrm2(cublasHandle_t h, int n, const double *x, double *out) {
  return cublasDnrm2(h, n, x, 1, out);
}
inline cublasStatus_t bl_nrm2(cublasHandle_t h, int n, const float *x, double *out) {
  float f = 0.0f;
  const cublasStatus_t st = cublasSnrm2(h, n, x, 1, &f);
  *out = f;
  return st;
}
inline cublasStatus_t bl_scal(cublasHandle_t h, int n, double a, double *x) { return cublasDscal(h, n, &a, x, 1); }
inline cublasStatus_t bl_scal(cublasHandle_t h, int n, double a, float *x) {
  const float f = (float)a;
  return cublasSscal(h, n, &f, x, 1);
}
inline cublasStatus_t bl_gemm(cublasHandle_t h, int m, int n, int k, const double *A, int lda, const double *B,
                              int ldb, double *C, int ldc) {
  const double one = 1.0, zero = 0.0;
  return cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, A, lda, B, ldb, &zero, C, ldc);
}

// The middle matrix's factorization starts from Q = P = I and Bd = [B 0; 0 0]
// (beta_k = 0 between B and the zero block).
template <typename T>
bdu_status thin_reset_core(bdu_thin_ctx *t) {
  bdu_ctx *h = t->core;
  const int64_t N = t->k + 1;
  cudaStream_t s = h->stream;
  cublasHandle_t cb = (cublasHandle_t)h->cublas;
  cudaError_t ce = cudaMemsetAsync(h->Q, 0, sizeof(T) * N * N, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->P, 0, sizeof(T) * N * N, s);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "rank-k step: resetting the middle factors");
  if (bl_copy(cb, (int)N, (const T *)t->ones, 1, (T *)h->Q, (int)N + 1) != CUBLAS_STATUS_SUCCESS ||
      bl_copy(cb, (int)N, (const T *)t->ones, 1, (T *)h->P, (int)N + 1) != CUBLAS_STATUS_SUCCESS)
    return fail(h, BDU_ECUDA, "rank-k step: cuBLAS copy failed");
  std::vector<double> hb(band_doubles(N, N), 0.0);
  BandPtrs hp = band_ptrs(hb.data(), N, N);
  hp.r1[1] = t->d[0];
  hp.r1[2] = t->k > 1 ? t->e[0] : 0.0;
  for (int64_t i = 2; i <= t->k; i++) hp.dg[2][i] = t->d[i - 1];
  for (int64_t i = 2; i <= t->k - 1; i++) hp.dg[3][i] = t->e[i - 1];
  ce = cudaMemcpyAsync(h->band, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  return ce == cudaSuccess ? BDU_OK : cuda_fail(h, ce, "rank-k step: resetting the middle band");
}

// Eq. defup and Eq. qrlr for one side: w[0:k] = X^T b (two Gram-Schmidt
// passes, accumulated), the remainder's norm delta into u[k] (FP64, with
// u[0:k] = w), and the unit remainder into column k of X (len x (k+1)); when
// b lies in span(X) the fixed fill vector is orthogonalized instead and
// delta = 0.
template <typename T>
bdu_status thin_side(bdu_thin_ctx *t, T *X, int64_t len, const T *b, const T *fill, T *w, double *u, int which,
                     bool *in_span) {
  bdu_ctx *h = t->core;
  cublasHandle_t cb = (cublasHandle_t)h->cublas;
  const int L = (int)len, k = (int)t->k;
  const T one = 1, zero = 0, mone = -1;
  T *r = (T *)t->r, *h1 = (T *)t->h1;
  auto ok = [](cublasStatus_t st) { return st == CUBLAS_STATUS_SUCCESS; };
  auto cgs2 = [&](const T *src, T *proj) {
    return ok(bl_gemv(cb, CUBLAS_OP_T, L, k, &one, X, L, src, &zero, h1)) && ok(bl_copy(cb, L, src, 1, r, 1)) &&
           ok(bl_gemv(cb, CUBLAS_OP_N, L, k, &mone, X, L, h1, &one, r)) &&
           ok(bl_gemv(cb, CUBLAS_OP_T, L, k, &one, X, L, r, &zero, proj)) &&
           ok(bl_gemv(cb, CUBLAS_OP_N, L, k, &mone, X, L, proj, &one, r)) && ok(bl_axpy(cb, k, &one, h1, proj));
  };
  double nb = 0.0, dl = 0.0;
  if (!cgs2(b, w) || !ok(bl_nrm2(cb, L, b, &nb)) || !ok(bl_nrm2(cb, L, r, &dl)))
    return fail(h, BDU_ECUDA, "rank-k step: cuBLAS projection failed");
  T *col = X + (size_t)k * len;
  *in_span = !(dl > (sizeof(T) == 8 ? kThinTau64 : kThinTau32) * nb);
  double scale_norm = dl;
  if (*in_span) {
    dl = 0.0;
    if (!cgs2(fill, (T *)t->h2) || !ok(bl_nrm2(cb, L, r, &scale_norm)))
      return fail(h, BDU_ECUDA, "rank-k step: cuBLAS projection failed");
    if (!(scale_norm > 0.0)) return fail(h, BDU_EINTERNAL, "rank-k step: no direction left outside the subspace");
  }
  if (!ok(bl_copy(cb, L, r, 1, col, 1)) || !ok(bl_scal(cb, L, 1.0 / scale_norm, col)))
    return fail(h, BDU_ECUDA, "rank-k step: cuBLAS scaling failed");
  cudaError_t ce = cudaSuccess;
  if (sizeof(T) == 4) ce = launch_convert_f32_to_f64((const float *)w, u, k, h->stream);
  t->delta_host[which] = dl;
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(u + k, &t->delta_host[which], sizeof(double), cudaMemcpyHostToDevice, h->stream);
  return ce == cudaSuccess ? BDU_OK : cuda_fail(h, ce, "rank-k step: staging delta");
}

template <typename T>
bdu_status thin_step(bdu_thin_ctx *t, int64_t *dropped, double *err2) {
  bdu_ctx *h = t->core;
  const int64_t m = t->m, n = t->n, k = t->k, N = k + 1;
  cudaStream_t s = h->stream;
  cublasHandle_t cb = (cublasHandle_t)h->cublas;
  if (cublasSetStream(cb, s) != CUBLAS_STATUS_SUCCESS ||
      cublasSetPointerMode(cb, CUBLAS_POINTER_MODE_HOST) != CUBLAS_STATUS_SUCCESS ||
      cublasSetMathMode(cb, CUBLAS_PEDANTIC_MATH) != CUBLAS_STATUS_SUCCESS)
    return fail(h, BDU_ECUDA, "rank-k step: cuBLAS set-up failed");
  bool sb = false, sc = false;
  bdu_status st = thin_side<T>(t, (T *)t->Qb, m, (const T *)t->x, (const T *)t->zq, (T *)t->wq, t->u, 0, &sb);
  if (st == BDU_OK) st = thin_side<T>(t, (T *)t->Pb, n, (const T *)t->y, (const T *)t->zp, (T *)t->wp, t->v, 1, &sc);
  if (st == BDU_OK) st = thin_reset_core<T>(t);
  if (st != BDU_OK) return st;
  // Algorithm 2 on the middle matrix (Eq. equivlrup): u = I^T u, v = I^T v exactly
  st = bdu_update_dev(h, t->u, t->v, 1);
  if (st != BDU_OK) return st;
  std::vector<double> d2(N), e2(N);
  cudaError_t ce = read_bidiagonal(h, d2.data(), e2.data());
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "rank-k step: reading the middle bidiagonal");
  // the index of the smallest column norm alpha_i^2 + beta_{i-1}^2 (ties: the last)
  int64_t drop = 0;
  double wmin = 0.0;
  for (int64_t i = 0; i < N; i++) {
    volatile double a2 = d2[i] * d2[i];
    double w = a2;
    if (i > 0) {
      volatile double b2 = e2[i - 1] * e2[i - 1];
      w = a2 + b2;
    }
    if (i == 0 || w <= wmin) {
      wmin = w;
      drop = i;
    }
  }
  volatile double er = d2[drop] * d2[drop];
  double err = er;
  if (drop > 0) {
    volatile double t2 = e2[drop - 1] * e2[drop - 1];
    err = err + t2;
  }
  if (drop < k) {
    volatile double t3 = e2[drop] * e2[drop];
    err = err + t3;
  }
  // [X, column] X2(:, kept) for X2 = Q2, P2 (Eq. bdlrup), into the spare buffer
  T *K2 = (T *)t->K2;
  for (int side = 0; side < 2; side++) {
    const T *X2 = (const T *)(side == 0 ? h->Q : h->P);
    if (drop > 0) ce = cudaMemcpyAsync(K2, X2, sizeof(T) * N * drop, cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess && drop < k)
      ce = cudaMemcpyAsync(K2 + N * drop, X2 + N * (drop + 1), sizeof(T) * N * (k - drop), cudaMemcpyDeviceToDevice, s);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "rank-k step: gathering the kept columns");
    const int64_t len = side == 0 ? m : n;
    T *Xb = (T *)(side == 0 ? t->Qb : t->Pb), *Xn = (T *)(side == 0 ? t->Qn : t->Pn);
    if constexpr (sizeof(T) == 4) {
      // mixed form: 3xTF32 on the tensor cores from K-contiguous copies, X^T
      // (leading dimension Np = N rounded up to a multiple of 4) in W and the
      // kept columns in E
      const int64_t Np = (N + 3) / 4 * 4;
      ce = launch_transpose32((const float *)Xb, len, (int)N, t->W, Np, s);
      if (ce == cudaSuccess) ce = launch_pad_copy32((const float *)K2, N, (int)k, t->E, Np, s);
      if (ce == cudaSuccess)
        ce = launch_gemm_tc(3, t->W, Np, t->E, Np, (int)len, (int)k, (int)N, (float *)Xn, 1, len, 1.0f, 0, h->status,
                            s);
      if (ce != cudaSuccess) return cuda_fail(h, ce, "rank-k step: the product with the kept columns");
    } else {
      if (bl_gemm(cb, (int)len, (int)k, (int)N, Xb, (int)len, K2, (int)N, Xn, (int)len) != CUBLAS_STATUS_SUCCESS)
        return fail(h, BDU_ECUDA, "rank-k step: cuBLAS GEMM failed");
    }
  }
  std::swap(t->Qb, t->Qn);
  std::swap(t->Pb, t->Pn);
  if (sizeof(T) == 4) {
    // FP32 factors: one Newton-Schulz step each, X <- X - X (X^T X - I) / 2
    ce = launch_reorth32((float *)t->Qb, m, (int)k, t->E, t->W, h->status, s);
    if (ce == cudaSuccess) ce = launch_reorth32((float *)t->Pb, n, (int)k, t->E, t->W, h->status, s);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "rank-k step: re-orthogonalization");
  }
  // B+ = Bbar+(kept, kept): the superdiagonal entry across the removed index is zero
  std::vector<double> dn, en;
  for (int64_t i = 0; i < N; i++)
    if (i != drop) dn.push_back(d2[i]);
  for (int64_t i = 0; i + 1 < N; i++) {
    if (i == drop || i + 1 == drop) continue;
    en.push_back(e2[i]);
  }
  if (drop > 0 && drop < k) en.insert(en.begin() + (drop - 1), 0.0);
  t->d = dn;
  t->e = en;
  t->e.resize(k > 1 ? k - 1 : 0);
  t->updates++;
  t->in_span_b += sb;
  t->in_span_c += sc;
  if (dropped) *dropped = drop;
  if (err2) *err2 = err;
  ce = cudaStreamSynchronize(s);
  return ce == cudaSuccess ? BDU_OK : cuda_fail(h, ce, "rank-k step");
}

template <typename T>
void thin_fill_host(std::vector<T> &z, std::vector<T> &ones, int64_t L, int64_t N) {
  // the fill vector z_i = frac(i * golden) - 0.5 (each step one IEEE operation)
  z.resize(L);
  for (int64_t i = 0; i < L; i++) {
    const double a = (double)i * kGolden;
    z[i] = (T)((a - floor(a)) - 0.5);
  }
  ones.assign(N, (T)1);
}

}  // namespace

extern "C" {

bdu_status bdu_thin_create(bdu_thin_handle *out, int64_t m, int64_t n, int64_t k, const double *Q1, const double *d,
                           const double *e, const double *P1, const bdu_options *opt) {
  if (!out) return fail(nullptr, BDU_EINVAL, "bdu_thin_create: output handle pointer is NULL");
  *out = nullptr;
  if (k < 1 || k >= m || k >= n || k > 16383)
    return fail(nullptr, BDU_EINVAL, "bdu_thin_create: need 1 <= k < min(m, n), k < 16384 (m=%lld n=%lld k=%lld)",
                (long long)m, (long long)n, (long long)k);
  if (m > (1LL << 24) || n > (1LL << 24) || m * (k + 1) > (1LL << 31) || n * (k + 1) > (1LL << 31))
    return fail(nullptr, BDU_EINVAL, "bdu_thin_create: factors too large for one GEMM call");
  if (!Q1 || !d || !P1 || (k > 1 && !e)) return fail(nullptr, BDU_EINVAL, "bdu_thin_create: NULL input pointer");
  bdu_options o;
  bdu_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != BDU_FP64 && o.precision != BDU_MIXED)
    return fail(nullptr, BDU_EINVAL, "bdu_thin_create: unknown precision %d", o.precision);
  // the middle matrix's factors start from the identity at every step: no
  // overlap, no checks or re-orthogonalization of them
  o.overlap = 0;
  o.reorth_every = 0;
  o.reorth_tol = 0.0;
  o.check_every = 0;
  if (!all_finite(Q1, m * k) || !all_finite(P1, n * k) || !all_finite(d, k) || (k > 1 && !all_finite(e, k - 1)))
    return fail(nullptr, BDU_EINVAL, "bdu_thin_create: non-finite value in Q1, d, e or P1");
  bdu_thin_ctx *t = new (std::nothrow) bdu_thin_ctx();
  if (!t) return fail(nullptr, BDU_ENOMEM, "bdu_thin_create: host allocation failed");
  t->m = m; t->n = n; t->k = k;
  t->mixed = o.precision == BDU_MIXED;
  t->d.assign(d, d + k);
  t->e.assign(k > 1 ? e : d, k > 1 ? e + (k - 1) : d);
  const int64_t N = k + 1;
  std::vector<double> eye(N * N, 0.0), dpad(N, 0.0), epad(N, 0.0);
  for (int64_t i = 0; i < N; i++) eye[i * N + i] = 1.0;
  for (int64_t i = 0; i < k; i++) dpad[i] = d[i];
  for (int64_t i = 0; i + 1 < k; i++) epad[i] = e[i];
  bdu_status st = bdu_create(&t->core, N, N, eye.data(), dpad.data(), epad.data(), eye.data(), &o);
  if (st != BDU_OK) {
    delete t;
    return st;
  }
  bdu_ctx *h = t->core;
  cublasHandle_t hb = nullptr;
  if (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) {
    bdu_destroy(h);
    delete t;
    return fail(nullptr, BDU_ENOMEM, "bdu_thin_create: cublasCreate failed");
  }
  h->cublas = hb;
  const size_t es = t->mixed ? sizeof(float) : sizeof(double);
  const int64_t L = m > n ? m : n;
  t->Qb = dev_alloc(h, es * m * N);
  t->Qn = dev_alloc(h, es * m * N);
  t->Pb = dev_alloc(h, es * n * N);
  t->Pn = dev_alloc(h, es * n * N);
  t->x = dev_alloc(h, es * m);
  t->y = dev_alloc(h, es * n);
  t->r = dev_alloc(h, es * L);
  t->zq = dev_alloc(h, es * m);
  t->zp = dev_alloc(h, es * n);
  t->h1 = dev_alloc(h, es * N);
  t->h2 = dev_alloc(h, es * N);
  t->ones = dev_alloc(h, es * N);
  t->K2 = dev_alloc(h, es * N * k);
  t->u = (double *)dev_alloc(h, sizeof(double) * N);
  t->v = (double *)dev_alloc(h, sizeof(double) * N);
  bool ok = t->Qb && t->Qn && t->Pb && t->Pn && t->x && t->y && t->r && t->zq && t->zp && t->h1 && t->h2 &&
            t->ones && t->K2 && t->u && t->v;
  if (t->mixed) {
    t->wq = dev_alloc(h, es * N);
    t->wp = dev_alloc(h, es * N);
    t->xd = (double *)dev_alloc(h, sizeof(double) * (L * k > m + n ? L * k : m + n));  // b and c, or a factor
    size_t ef = 0, wf = 0;
    reorth32_workspace(L, (int)(k + 1), &ef, &wf);  // also the products' operand copies (k + 1 columns)
    t->E = (float *)dev_alloc(h, sizeof(float) * ef);
    t->W = (float *)dev_alloc(h, sizeof(float) * wf);
    ok = ok && t->wq && t->wp && t->xd && t->E && t->W;
  } else {
    t->wq = t->u;
    t->wp = t->v;
  }
  if (!ok) {
    bdu_destroy(h);
    delete t;
    return fail(nullptr, BDU_ENOMEM, "bdu_thin_create: device allocation failed");
  }
  cudaStream_t s = h->stream;
  cudaError_t ce = cudaSuccess;
  std::vector<double> zd, od;
  std::vector<float> zf, of;
  if (t->mixed) {
    thin_fill_host<float>(zf, of, L, N);
    ce = cudaMemcpyAsync(t->xd, Q1, sizeof(double) * m * k, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = launch_convert_f64_to_f32(t->xd, (float *)t->Qb, m * k, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->xd, P1, sizeof(double) * n * k, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = launch_convert_f64_to_f32(t->xd, (float *)t->Pb, n * k, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->zq, zf.data(), es * m, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->zp, zf.data(), es * n, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->ones, of.data(), es * N, cudaMemcpyHostToDevice, s);
  } else {
    thin_fill_host<double>(zd, od, L, N);
    ce = cudaMemcpyAsync(t->Qb, Q1, sizeof(double) * m * k, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->Pb, P1, sizeof(double) * n * k, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->zq, zd.data(), es * m, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->zp, zd.data(), es * n, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->ones, od.data(), es * N, cudaMemcpyHostToDevice, s);
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    fail(nullptr, BDU_ECUDA, "bdu_thin_create: %s", cudaGetErrorString(ce));
    bdu_destroy(h);
    delete t;
    return BDU_ECUDA;
  }
  *out = t;
  return BDU_OK;
}

static bdu_status thin_update_common(bdu_thin_handle t, const double *b, const double *c, bool host,
                                     int64_t *dropped, double *err2) {
  if (!t) return fail(nullptr, BDU_EINVAL, "NULL handle");
  bdu_ctx *h = t->core;
  ThinGuard g(t);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  if (h->poisoned) return fail(h, BDU_EPOISONED, "handle poisoned by an earlier failure: %s", h->err);
  if (!b || !c) return fail(h, BDU_EINVAL, "NULL update vector");
  if (host && (!all_finite(b, t->m) || !all_finite(c, t->n))) return fail(h, BDU_EINVAL, "non-finite value in b or c");
  cudaError_t ce = cudaSetDevice(h->device);
  cudaStream_t s = h->stream;
  const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (!t->mixed) {
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->x, b, sizeof(double) * t->m, kind, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->y, c, sizeof(double) * t->n, kind, s);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "rank-k step: staging b, c");
    return thin_step<double>(t, dropped, err2);
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->xd, b, sizeof(double) * t->m, kind, s);
  if (ce == cudaSuccess) ce = launch_convert_f64_to_f32(t->xd, (float *)t->x, t->m, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->xd + t->m, c, sizeof(double) * t->n, kind, s);
  if (ce == cudaSuccess) ce = launch_convert_f64_to_f32(t->xd + t->m, (float *)t->y, t->n, s);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "rank-k step: staging b, c");
  return thin_step<float>(t, dropped, err2);
}

bdu_status bdu_thin_update(bdu_thin_handle t, const double *b, const double *c, int64_t *dropped, double *err2) {
  return thin_update_common(t, b, c, true, dropped, err2);
}

bdu_status bdu_thin_update_dev(bdu_thin_handle t, const double *db, const double *dc, int64_t *dropped,
                               double *err2) {
  return thin_update_common(t, db, dc, false, dropped, err2);
}

bdu_status bdu_thin_read(bdu_thin_handle t, double *Q1, double *d, double *e, double *P1) {
  if (!t) return fail(nullptr, BDU_EINVAL, "NULL handle");
  bdu_ctx *h = t->core;
  ThinGuard g(t);
  if (!g.ok) return fail(h, BDU_EBUSY, "handle in use by another thread");
  cudaSetDevice(h->device);
  cudaStream_t s = h->stream;
  cudaError_t ce = cudaSuccess;
  for (int side = 0; side < 2 && ce == cudaSuccess; side++) {
    double *dst = side == 0 ? Q1 : P1;
    if (!dst) continue;
    const int64_t cnt = (side == 0 ? t->m : t->n) * t->k;
    const void *src = side == 0 ? t->Qb : t->Pb;
    if (t->mixed) {
      ce = launch_convert_f32_to_f64((const float *)src, t->xd, cnt, s);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(dst, t->xd, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s);
    } else {
      ce = cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  }
  if (ce != cudaSuccess) return cuda_fail(h, ce, "bdu_thin_read");
  if (d) std::copy(t->d.begin(), t->d.end(), d);
  if (e) std::copy(t->e.begin(), t->e.end(), e);
  return BDU_OK;
}

bdu_status bdu_thin_stats(bdu_thin_handle t, int64_t *updates, int64_t *in_span_b, int64_t *in_span_c) {
  if (!t) return fail(nullptr, BDU_EINVAL, "NULL handle");
  if (updates) *updates = t->updates;
  if (in_span_b) *in_span_b = t->in_span_b;
  if (in_span_c) *in_span_c = t->in_span_c;
  return BDU_OK;
}

const char *bdu_thin_last_error(bdu_thin_handle t) { return t ? t->core->err : t_create_err; }

void bdu_thin_destroy(bdu_thin_handle t) {
  if (!t) return;
  bdu_destroy(t->core);
  delete t;
}

}  // extern "C"
