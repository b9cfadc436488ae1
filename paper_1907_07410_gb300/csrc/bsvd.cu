// C ABI of libbsvd: context, argument checks, buffers and the order of
// kernel launches for each call. See include/bsvd.h for the contract.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>

#include "bsvd.h"
#include "kernels.h"

// Longest the host polls for a step's convergence counters before it falls
// back to a stream synchronisation.
static constexpr int kPollMs = 50;

using namespace bsvd;

namespace {

// A device allocation that only grows.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t want) {
    if (want <= bytes && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (want == 0) want = 16;
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T *as() const { return static_cast<T *>(p); }
};

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType,
                                  cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up through the runtime.
EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

struct bsvd_ctx {
  bsvd_config cfg;
  cudaStream_t st = nullptr;
  std::string err;
  int device = 0;

  // partition
  bool parted = false;
  int64_t m = 0, n = 0, nnz = 0;
  int32_t p = 0, q = 0, nblocks = 0;
  std::vector<int64_t> rb, cb;
  bool eq_r = true, eq_c = true, has_rperm = false, has_cperm = false;
  bool diag = false;        // block-diagonal batch of independent blocks
  int64_t br = 0, bc = 0;
  std::vector<BlockMeta> meta;
  // blocks this context holds (bsvd_set_owned); empty: all of them
  std::vector<uint8_t> own;
  int64_t arena = 0;
  DevBuf d_rb, d_cb, d_rperm, d_cperm, d_seen, d_meta, d_counts, d_sums,
      d_maxabs, d_mu, d_W, d_err;
  // bf16 [Y; M] planes, per-block shift and delta, TMA maps (tensor Gram)
  bool tc_planes = false, tc_exact = false;
  // the float32 arena W is written unless the BF16 form's tensor-core
  // projection reads the bf16 copy instead
  bool w32 = true;
  int32_t gram_used = 0;    // 1: FP32 SIMT, 2: exact tensor, 3: tf32, 4: bf16
  DevBuf d_VX, d_shift, d_delta, d_maps, d_flag;
  DevBuf d_wmaps;           // TMA maps over the float32 blocks (tf32 Gram)

  // factor
  bool factored = false;
  int32_t k = 0, bsub = 0, kp = 4;
  DevBuf d_G, d_X, d_Z, d_SH, d_RP, d_T, d_theta, d_state, d_Fs, d_FL, d_sigma,
      d_running, d_gtiles, d_rowtiles, d_ltiles, d_finv, d_chunks;
  int32_t n_gtiles = 0, n_rowtiles = 0, n_ltiles = 0;
  // tensor-core panel products: 128-row tiles and one TMA map per block of G
  DevBuf d_ptiles, d_gmaps, d_xmaps;
  DevBuf d_XB, d_ZB;         // B forms of the panels X, Z (2 s_pad x B floats)
  // pinned and mapped: running count, largest degree, sequence number
  int32_t *h_run = nullptr;
  int32_t *d_run_host = nullptr;  // the same memory seen from the device
  int32_t run_seq = 0;
  int32_t n_ptiles = 0;
  std::vector<CUtensorMap> h_gmaps, h_xmaps, h_pwmaps;
  // tensor-core projection: 128-column tiles of W and one TMA map per block
  DevBuf d_pjtiles, d_pwmaps;
  int32_t n_pjtiles = 0;
  int32_t n_chunks = 0;      // kChunkRows-row chunks of the panels
  // finalisation: per-tile column statistics of F_L and F_s, column flips
  DevBuf d_lpart, d_spart, d_flip;
  // the persistent panel products' tile counter, and the CTAs they launch
  DevBuf d_pctl;
  int32_t nsm = 1;
  // panel products' device time: [0] summed launch durations (ns), [1] the
  // running launch's start; the graph loop's step counter
  DevBuf d_ptime, d_loopctl;
  // the device-driven form: the captured graph, the layout key it was built
  // for, the key of this and of the previous factorisation, kernel counts
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap = nullptr, side = nullptr, side2 = nullptr;  // capture
  // bsvd_partition_quantile uploads x on its own stream while the grid is
  // cut on the caller's
  cudaStream_t up = nullptr;
  cudaEvent_t ev_up_fork = nullptr, ev_up_join = nullptr;
  std::vector<unsigned char> gkey_now, gkey_prev, gkey_exec;
  bool graph_failed = false, capturing = false;
  std::string graph_err;     // why the graph could not be built
  int64_t graph_static_launches = 0, graph_loop_launches = 0;
  int32_t last_graph = 0;   // last factor's loop: 0 none, 1 host, 2 graph
  int64_t panel_launches = 0;   // tensor-core panel products, last factor
  // the BF16 form's projection: maps over the bf16 blocks and over F_s's
  // bf16 B form, and that B form
  DevBuf d_pbmaps, d_fbmaps, d_FB;
  std::vector<CUtensorMap> h_pbmaps, h_fbmaps;
  // the layout the uploaded tables and tensor maps were built for (see
  // factor_impl), and the solver's initial state kept on the device
  std::vector<unsigned char> fsig;
  DevBuf d_state0;

  // blocked SGD (Algorithms 1-2): ratings in epoch order, block ranges,
  // schedule, model
  bool sgd_ready = false, sgd_trained = false;
  int64_t sgd_nnz = 0;
  int32_t sgd_k = 0;
  DevBuf d_sgd_cnt, d_sgd_off, d_sgd_key, d_sgd_src, d_sgd_u, d_sgd_i,
      d_sgd_x, d_sgd_r, d_sgd_c, d_sgd_range, d_sgd_blocks, d_sgd_P,
      d_sgd_Q, d_sgd_bu, d_sgd_bi, d_sgd_sum, d_sgd_P32, d_sgd_Q32;
  std::vector<int32_t> sgd_step_off;   // steps: blocks [off[s], off[s+1])
  bool any_capped = false;

  // staging of host arguments and results
  DevBuf s_a, s_b, s_c, s_out, d_partials, d_rmse;
  // activity-quantile cut: counts, sort keys, running sums, perms, bounds
  DevBuf d_qcnt, d_qkeys, d_qcum, d_qperm, d_qbounds;
  DevBuf d_qperm2;          // the columns' permutation (partition_quantile)

  // tracing: kernel launch count and per-phase CUDA events
  int64_t launches = 0;
  cudaEvent_t ev[10] = {};
  double phase_ms[8] = {};

  GridDesc grid() const {
    GridDesc g;
    g.m = m; g.n = n; g.p = p; g.q = q;
    g.equal_rows = eq_r ? 1 : 0;
    g.equal_cols = eq_c ? 1 : 0;
    g.diag = diag ? 1 : 0;
    g.pad = 0;
    g.br = br; g.bc = bc;
    g.row_bounds = d_rb.as<int64_t>();
    g.col_bounds = d_cb.as<int64_t>();
    g.row_perm = has_rperm ? d_rperm.as<int32_t>() : nullptr;
    g.col_perm = has_cperm ? d_cperm.as<int32_t>() : nullptr;
    return g;
  }
};

namespace {

bsvd_status fail(bsvd_ctx *c, bsvd_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c->err = buf;
  return s;
}

bsvd_status cuda_fail(bsvd_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, BSVD_ENOMEM, "%s: out of device memory", what);
  }
  return fail(c, BSVD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

bool is_device_ptr(const void *ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller array: the pointer itself when it is device
// memory, else a copy in the staging buffer.
cudaError_t device_view(bsvd_ctx *c, const void *ptr, size_t bytes,
                        DevBuf &stage, const void **out) {
  if (bytes == 0 || is_device_ptr(ptr)) {
    *out = ptr;
    return cudaSuccess;
  }
  cudaError_t e = stage.ensure(bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(stage.p, ptr, bytes, cudaMemcpyHostToDevice, c->st);
  *out = stage.p;
  return e;
}

bsvd_status read_errors(bsvd_ctx *c, const char *what) {
  int32_t h = 0;
  CK(cudaMemcpyAsync(&h, c->d_err.p, sizeof h, cudaMemcpyDeviceToHost, c->st),
     what);
  CK(cudaStreamSynchronize(c->st), what);
  if (h) {
    std::string msg = std::string(what) + ":";
    if (h & kErrIndex) msg += " id out of range or off the block diagonal;";
    if (h & kErrValue) msg += " non-finite rating or |x| >= 2^31;";
    if (h & kErrSumRange) msg += " ratings too large for exact block sums;";
    if (h & kErrBadPerm) msg += " invalid permutation;";
    if (h & kErrTimeout) msg += " a device-side wait timed out;";
    CK(cudaMemsetAsync(c->d_err.p, 0, sizeof(int32_t), c->st), what);
    return fail(c, (h & kErrTimeout) ? BSVD_ETIMEOUT : BSVD_EINVAL, "%s",
                msg.c_str());
  }
  return BSVD_OK;
}

// Phase events: mark(i) records event i on the stream when profiling.
void mark(bsvd_ctx *c, int i) {
  if (!c->cfg.profile || !c->ev[i]) return;
  if (c->capturing)   // an event-record node of the graph
    cudaEventRecordWithFlags(c->ev[i], c->st, cudaEventRecordExternal);
  else
    cudaEventRecord(c->ev[i], c->st);
}

// After a synchronised call: phase_ms[ph] = time between events a and b.
void take(bsvd_ctx *c, int ph, int a, int b) {
  if (!c->cfg.profile) return;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) == cudaSuccess)
    c->phase_ms[ph] = ms;
  else
    cudaGetLastError();
}

bool bounds_ok(const int64_t *b, int32_t parts, int64_t total) {
  if (b[0] != 0 || b[parts] != total) return false;
  for (int32_t j = 0; j < parts; ++j)
    if (b[j + 1] < b[j]) return false;
  return true;
}

int32_t subspace_width(int32_t k, int32_t oversample) {
  int32_t extra = oversample > 0 ? oversample : std::max(8, k / 2);
  int32_t want = k + extra;
  if (want <= 16) return 16;
  if (want <= 32) return 32;
  return 64;
}

// The panel products' device timer: no time summed yet, no launch running.
cudaError_t reset_ptime(bsvd_ctx *c) {
  cudaError_t e = cudaMemsetAsync(c->d_ptime.p, 0,
                                  3 * sizeof(unsigned long long), c->st);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(c->d_ptime.as<unsigned long long>() + 1, 0xFF,
                         sizeof(unsigned long long), c->st);
}

// Capture one factorisation into c->gexec: pre, then a conditional WHILE
// node whose body is one Rayleigh-Ritz step, k_loopctl (which sets the
// condition from the number of blocks still iterating) and one full-degree
// filter, then post. The body is captured on a second stream into the
// node's body graph. Kernel counts: graph_static_launches per graph launch
// outside the loop, graph_loop_launches per loop step.
template <class Pre, class Rr, class Step, class Prod, class Post>
cudaError_t build_graph(bsvd_ctx *c, Pre &pre, Rr &rr, Step &fstep,
                        Prod &fprod, Post &post) {
  cudaGraph_t g = nullptr;
  cudaError_t r = cudaGraphCreate(&g, 0);
  if (r != cudaSuccess) return r;
  // capture on the context's own streams (the caller's stream may be the
  // legacy default stream, which cannot be captured); the graph is then
  // launched on the caller's stream
  for (cudaStream_t *sp : {&c->cap, &c->side, &c->side2}) {
    if (!*sp) {
      r = cudaStreamCreateWithFlags(sp, cudaStreamNonBlocking);
      if (r != cudaSuccess) {
        cudaGraphDestroy(g);
        return r;
      }
    }
  }
  const cudaStream_t user_st = c->st;
  const cudaStream_t st = c->cap;
  c->st = st;
  const int64_t l0 = c->launches;
  int64_t l1 = 0, l2 = 0;
  c->capturing = true;
  // the first failing step names itself in graph_err
  auto note = [&](const char *what, cudaError_t e) {
    if (e != cudaSuccess && c->graph_err.empty())
      c->graph_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e;
  };
  r = note("begin capture", cudaStreamBeginCaptureToGraph(
                                st, g, nullptr, nullptr, 0,
                                cudaStreamCaptureModeThreadLocal));
  const bool main_open = r == cudaSuccess;
  if (r == cudaSuccess) r = note("Gram and start", pre());
  if (r == cudaSuccess)
    r = note("loop counter", cudaMemsetAsync(c->d_loopctl.p, 0,
                                              2 * sizeof(int32_t), st));
  if (r == cudaSuccess) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaGraph_t cg = nullptr;
    r = note("capture info", cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg,
                                                      &deps, nullptr, &nd));
    cudaGraphConditionalHandle h = 0;
    if (r == cudaSuccess)
      r = note("conditional handle",
               cudaGraphConditionalHandleCreate(&h, cg, 1,
                                                cudaGraphCondAssignDefault));
    // zeroed storage: the struct's union has no default constructor
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    std::memset(npbuf, 0, sizeof npbuf);
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(npbuf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (r == cudaSuccess)
      r = note("conditional node",
               cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &np));
    if (r == cudaSuccess)
      r = note("capture dependencies",
               cudaStreamUpdateCaptureDependencies(
                   st, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    if (r == cudaSuccess) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      c->st = c->side;
      l1 = c->launches;
      r = note("begin body capture",
               cudaStreamBeginCaptureToGraph(c->side, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
      if (r == cudaSuccess) {
        // filter steps 3 .. cheb_degree each sit in an IF node that
        // k_loopctl opens when some running block's degree reaches the step
        const int deg = c->cfg.cheb_degree;
        LoopHandles lh;
        std::memset(&lh, 0, sizeof lh);
        lh.first = 3;
        lh.n = deg >= 3 ? deg - 2 : 0;
        cudaError_t rb = cudaSuccess;
        for (int j = 0; j < lh.n && rb == cudaSuccess; ++j)
          rb = note("step handle", cudaGraphConditionalHandleCreate(
                                       &lh.h[j], body, 0,
                                       cudaGraphCondAssignDefault));
        if (rb == cudaSuccess) rb = note("Rayleigh-Ritz step", rr());
        if (rb == cudaSuccess) {
          rb = note("loop control",
                    launch_loopctl(c->d_running.as<int32_t>(),
                                   c->d_loopctl.as<int32_t>(),
                                   c->cfg.max_iters + 2, h, lh, c->side));
          ++c->launches;
        }
        for (int j = 1; j <= std::min(deg, 2) && rb == cudaSuccess; ++j)
          rb = note("filter step", fstep(j));
        for (int j = 3; j <= deg && rb == cudaSuccess; ++j) {
          cudaStreamCaptureStatus bs;
          const cudaGraphNode_t *bdeps = nullptr;
          size_t bnd = 0;
          cudaGraph_t bg = nullptr;
          rb = note("body capture info",
                    cudaStreamGetCaptureInfo(c->side, &bs, nullptr, &bg, &bdeps,
                                             nullptr, &bnd));
          alignas(cudaGraphNodeParams) unsigned char ibuf[sizeof(cudaGraphNodeParams)];
          std::memset(ibuf, 0, sizeof ibuf);
          cudaGraphNodeParams &ip = *reinterpret_cast<cudaGraphNodeParams *>(ibuf);
          ip.type = cudaGraphNodeTypeConditional;
          ip.conditional.handle = lh.h[j - 3];
          ip.conditional.type = cudaGraphCondTypeIf;
          ip.conditional.size = 1;
          cudaGraphNode_t inode = nullptr;
          if (rb == cudaSuccess)
            rb = note("step node",
                      cudaGraphAddNode(&inode, bg, bdeps, nullptr, bnd, &ip));
          if (rb == cudaSuccess)
            rb = note("body dependencies",
                      cudaStreamUpdateCaptureDependencies(
                          c->side, &inode, nullptr, 1,
                          cudaStreamSetCaptureDependencies));
          if (rb == cudaSuccess) {
            const cudaStream_t body_st = c->st;
            c->st = c->side2;
            rb = note("begin step capture",
                      cudaStreamBeginCaptureToGraph(
                          c->side2, ip.conditional.phGraph_out[0], nullptr,
                          nullptr, 0, cudaStreamCaptureModeThreadLocal));
            if (rb == cudaSuccess) {
              const cudaError_t rs = note("filter step", fstep(j));
              cudaGraph_t sout = nullptr;
              const cudaError_t re2 = note(
                  "end step capture", cudaStreamEndCapture(c->side2, &sout));
              rb = rs != cudaSuccess ? rs : re2;
            }
            c->st = body_st;
          }
        }
        if (rb == cudaSuccess) rb = note("product", fprod());
        cudaGraph_t bout = nullptr;
        const cudaError_t re =
            note("end body capture", cudaStreamEndCapture(c->side, &bout));
        r = rb != cudaSuccess ? rb : re;
      }
      l2 = c->launches;
      c->st = st;
    }
  }
  if (r == cudaSuccess) r = note("projection", post());
  c->st = user_st;
  if (main_open) {
    cudaGraph_t gout = nullptr;
    const cudaError_t re = note("end capture", cudaStreamEndCapture(st, &gout));
    if (r == cudaSuccess) r = re;
  }
  c->capturing = false;
  if (r != cudaSuccess && c->graph_err.empty())
    c->graph_err = std::string("capture: ") + cudaGetErrorString(r);
  if (r == cudaSuccess) {
    r = cudaGraphInstantiate(&c->gexec, g, 0);
    if (r != cudaSuccess)
      c->graph_err = std::string("instantiate: ") + cudaGetErrorString(r);
  }
  cudaGraphDestroy(g);
  const int64_t l3 = c->launches;
  c->launches = l0;                 // captured, not run
  // the filter steps inside IF nodes are counted as the loop opens them
  const int64_t cond = c->cfg.cheb_degree >= 3
                           ? (int64_t)(c->cfg.cheb_degree - 2) * (c->n_rowtiles > 0)
                           : 0;
  c->graph_loop_launches = l2 - l1 - cond;
  c->graph_static_launches = (l3 - l0) - (l2 - l1);
  return r;
}

}  // namespace

extern "C" {

void bsvd_config_default(bsvd_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->precision = BSVD_FP32;
  cfg->clamp = 0;
  cfg->clamp_lo = 1.0f;
  cfg->clamp_hi = 5.0f;
  cfg->oversample = 0;
  cfg->cheb_degree = 8;
  cfg->max_iters = 30;
  cfg->max_sweeps = 30;
  cfg->tol = 0.0;        // per precision, set by bsvd_create
  cfg->seed = 0x5eed5eedull;
  cfg->stream = nullptr;
  cfg->panel_path = 0;
  cfg->loop = 0;
}

bsvd_status bsvd_create(const bsvd_config *cfg, bsvd_ctx **out) {
  if (!out) return BSVD_EINVAL;
  *out = nullptr;
  bsvd_ctx *c = new (std::nothrow) bsvd_ctx();
  if (!c) return BSVD_ENOMEM;
  bsvd_config_default(&c->cfg);
  if (cfg) {
    c->cfg = *cfg;
    if (c->cfg.cheb_degree <= 0) c->cfg.cheb_degree = 8;
    if (c->cfg.max_iters <= 0) c->cfg.max_iters = 30;
    if (c->cfg.max_sweeps <= 0) c->cfg.max_sweeps = 30;
  }
  if (!(c->cfg.tol > 0))
    c->cfg.tol = c->cfg.precision == BSVD_FP32   ? 1e-5
                 : c->cfg.precision == BSVD_TF32 ? 1e-4
                                                 : 5e-4;
  if ((c->cfg.precision != BSVD_FP32 && c->cfg.precision != BSVD_TF32 &&
       c->cfg.precision != BSVD_BF16) ||
      c->cfg.gram_path < 0 ||
      c->cfg.gram_path > 2 || c->cfg.panel_path < 0 ||
      c->cfg.panel_path > 1 || c->cfg.loop < 0 || c->cfg.loop > 2 ||
      c->cfg.cheb_degree % 2 != 0 ||
      c->cfg.cheb_degree > 64 || (c->cfg.clamp && !(c->cfg.clamp_lo <= c->cfg.clamp_hi))) {
    delete c;
    return BSVD_EINVAL;
  }
  c->st = static_cast<cudaStream_t>(c->cfg.stream);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount,
                             c->device) != cudaSuccess ||
      c->d_err.ensure(sizeof(int32_t)) != cudaSuccess ||
      cudaMemsetAsync(c->d_err.p, 0, sizeof(int32_t), c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return BSVD_ECUDA;
  }
  if (c->cfg.profile) {
    for (auto &e : c->ev) {
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        e = nullptr;
      }
    }
  }
  *out = c;
  return BSVD_OK;
}

void bsvd_destroy(bsvd_ctx *c) {
  if (!c) return;
  DevBuf *bufs[] = {&c->d_rb, &c->d_cb, &c->d_rperm, &c->d_cperm, &c->d_seen,
                    &c->d_meta, &c->d_counts, &c->d_sums, &c->d_maxabs,
                    &c->d_mu, &c->d_W, &c->d_err, &c->d_G, &c->d_X, &c->d_Z,
                    &c->d_SH, &c->d_RP, &c->d_T, &c->d_theta, &c->d_state, &c->d_Fs,
                    &c->d_FL, &c->d_sigma, &c->d_running, &c->d_gtiles,
                    &c->d_rowtiles, &c->d_ltiles, &c->s_a, &c->s_b, &c->s_c,
                    &c->s_out, &c->d_partials, &c->d_rmse, &c->d_VX,
                    &c->d_shift, &c->d_delta, &c->d_maps, &c->d_flag,
                    &c->d_wmaps, &c->d_ptiles, &c->d_gmaps, &c->d_xmaps, &c->d_XB, &c->d_ZB,
                    &c->d_pjtiles, &c->d_pwmaps, &c->d_state0,
                    &c->d_sgd_cnt, &c->d_sgd_off, &c->d_sgd_key,
                    &c->d_sgd_src, &c->d_sgd_u, &c->d_sgd_i, &c->d_sgd_x,
                    &c->d_sgd_range, &c->d_sgd_blocks, &c->d_sgd_P,
                    &c->d_sgd_Q, &c->d_sgd_bu, &c->d_sgd_bi, &c->d_sgd_sum,
                    &c->d_sgd_r, &c->d_sgd_c, &c->d_sgd_P32, &c->d_sgd_Q32,
                    &c->d_qcnt, &c->d_qkeys, &c->d_qcum, &c->d_qperm,
                    &c->d_qperm2,
                    &c->d_qbounds, &c->d_pbmaps, &c->d_fbmaps, &c->d_FB,
                    &c->d_lpart, &c->d_spart, &c->d_flip, &c->d_pctl,
                    &c->d_ptime, &c->d_loopctl, &c->d_finv, &c->d_chunks};
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  if (c->up) cudaStreamSynchronize(c->up);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->side2) cudaStreamDestroy(c->side2);
  if (c->up) cudaStreamDestroy(c->up);
  if (c->ev_up_fork) cudaEventDestroy(c->ev_up_fork);
  if (c->ev_up_join) cudaEventDestroy(c->ev_up_join);
  for (DevBuf *b : bufs) b->release();
  for (auto &e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->h_run) cudaFreeHost(c->h_run);
  delete c;
}

const char *bsvd_last_error(const bsvd_ctx *c) {
  return c ? c->err.c_str() : "null context";
}

static bsvd_status partition_impl(bsvd_ctx *c, int64_t m, int64_t n,
                                  int64_t nnz, const int32_t *u,
                                  const int32_t *i, const float *x, int32_t p,
                                  int32_t q, const int64_t *row_bounds,
                                  const int64_t *col_bounds,
                                  const int32_t *row_perm,
                                  const int32_t *col_perm, bool diag) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  c->sgd_ready = false;      // a new grid invalidates the SGD order
  c->sgd_trained = false;
  if (m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX || nnz < 0)
    return fail(c, BSVD_EINVAL, "partition: bad sizes m=%lld n=%lld nnz=%lld",
                (long long)m, (long long)n, (long long)nnz);
  if (p < 1 || q < 1 || (!row_bounds && p > m) || (!col_bounds && q > n))
    return fail(c, BSVD_EINVAL, "partition: bad grid %d x %d", p, q);
  if (nnz > 0 && (!u || !i || !x))
    return fail(c, BSVD_EINVAL, "partition: null rating arrays");
  if ((int64_t)p * q > (int64_t)INT32_MAX)
    return fail(c, BSVD_EINVAL, "partition: too many blocks");
  if (row_bounds && !bounds_ok(row_bounds, p, m))
    return fail(c, BSVD_EINVAL, "partition: bad row bounds");
  if (col_bounds && !bounds_ok(col_bounds, q, n))
    return fail(c, BSVD_EINVAL, "partition: bad column bounds");
  if (!c->own.empty() && (int64_t)c->own.size() != (diag ? (int64_t)p : (int64_t)p * q))
    return fail(c, BSVD_EINVAL, "partition: the owned-block mask has %lld "
                "entries for %lld blocks", (long long)c->own.size(),
                (long long)(diag ? (int64_t)p : (int64_t)p * q));

  c->parted = false;
  c->factored = false;
  c->m = m; c->n = n; c->nnz = nnz; c->p = p; c->q = q;
  c->diag = diag;
  c->nblocks = diag ? p : p * q;
  c->eq_r = row_bounds == nullptr;
  c->eq_c = col_bounds == nullptr;
  c->br = (m + p - 1) / p;
  c->bc = (n + q - 1) / q;
  c->rb.assign(p + 1, 0);
  c->cb.assign(q + 1, 0);
  for (int32_t j = 0; j <= p; ++j)
    c->rb[j] = row_bounds ? row_bounds[j] : std::min<int64_t>(j * c->br, m);
  for (int32_t j = 0; j <= q; ++j)
    c->cb[j] = col_bounds ? col_bounds[j] : std::min<int64_t>(j * c->bc, n);

  // block shapes and the dense arena layout
  c->meta.assign(c->nblocks, BlockMeta());
  int64_t off = 0, vxoff = 0;
  for (int32_t bi = 0; bi < p; ++bi) {
    for (int32_t bj = 0; bj < q; ++bj) {
      if (diag && bi != bj) continue;
      BlockMeta &bm = c->meta[diag ? bi : bi * q + bj];
      std::memset(&bm, 0, sizeof bm);
      bm.mb = (int32_t)(c->rb[bi + 1] - c->rb[bi]);
      bm.nb = (int32_t)(c->cb[bj + 1] - c->cb[bj]);
      bm.trans = bm.nb <= bm.mb ? 1 : 0;
      bm.s = std::min(bm.mb, bm.nb);
      bm.L = std::max(bm.mb, bm.nb);
      bm.s_pad = (int32_t)round_up(bm.s, kPad);
      bm.L_pad = (int32_t)round_up(bm.L, kPad);
      bm.row0 = c->rb[bi];
      bm.col0 = c->cb[bj];
      const int32_t b = diag ? bi : bi * q + bj;
      bm.owned = c->own.empty() || c->own[b] ? 1 : 0;
      bm.w_off = off;
      bm.s128 = (int32_t)round_up(bm.s, 128);
      bm.vx_off = vxoff;
      if (!bm.owned) continue;   // another shard's block: no dense storage
      off += (int64_t)bm.s_pad * bm.L_pad;
      // exact Gram: planes [Y; M]; bf16 Gram: one bf16 copy of W
      vxoff += (c->cfg.precision == BSVD_BF16 ? 1 : 2) * (int64_t)bm.s128 *
               bm.L_pad;
    }
  }
  c->arena = off;

  const int32_t nb = c->nblocks;
  CK(c->d_rb.ensure(sizeof(int64_t) * (p + 1)), "partition");
  CK(c->d_cb.ensure(sizeof(int64_t) * (q + 1)), "partition");
  CK(c->d_meta.ensure(sizeof(BlockMeta) * nb), "partition");
  CK(c->d_counts.ensure(sizeof(unsigned long long) * nb), "partition");
  CK(c->d_sums.ensure(sizeof(long long) * nb), "partition");
  CK(c->d_maxabs.ensure(sizeof(unsigned int)), "partition");
  CK(c->d_mu.ensure(sizeof(float) * nb), "partition");
  c->w32 = !(c->cfg.precision == BSVD_BF16 && c->cfg.panel_path == 0);
  if (c->w32)
    CK(c->d_W.ensure(sizeof(float) * std::max<int64_t>(off, 1)), "partition");
  CK(cudaMemcpyAsync(c->d_rb.p, c->rb.data(), sizeof(int64_t) * (p + 1),
                     cudaMemcpyHostToDevice, c->st), "partition");
  CK(cudaMemcpyAsync(c->d_cb.p, c->cb.data(), sizeof(int64_t) * (q + 1),
                     cudaMemcpyHostToDevice, c->st), "partition");
  CK(cudaMemcpyAsync(c->d_meta.p, c->meta.data(), sizeof(BlockMeta) * nb,
                     cudaMemcpyHostToDevice, c->st), "partition");

  // permutations: copied into context memory, then checked on the device
  c->has_rperm = row_perm != nullptr;
  c->has_cperm = col_perm != nullptr;
  CK(cudaMemsetAsync(c->d_err.p, 0, sizeof(int32_t), c->st), "partition");
  if (row_perm) {
    CK(c->d_rperm.ensure(sizeof(int32_t) * m), "partition");
    CK(c->d_seen.ensure(sizeof(int32_t) * std::max(m, n)), "partition");
    CK(cudaMemcpyAsync(c->d_rperm.p, row_perm, sizeof(int32_t) * m,
                       cudaMemcpyDefault, c->st), "partition");
    CK(launch_perm_check(c->d_rperm.as<int32_t>(), m, c->d_seen.as<int32_t>(),
                         c->d_err.as<int32_t>(), c->st), "partition");
    c->launches += 2;
  }
  if (col_perm) {
    CK(c->d_cperm.ensure(sizeof(int32_t) * n), "partition");
    CK(c->d_seen.ensure(sizeof(int32_t) * std::max(m, n)), "partition");
    CK(cudaMemcpyAsync(c->d_cperm.p, col_perm, sizeof(int32_t) * n,
                       cudaMemcpyDefault, c->st), "partition");
    CK(launch_perm_check(c->d_cperm.as<int32_t>(), n, c->d_seen.as<int32_t>(),
                         c->d_err.as<int32_t>(), c->st), "partition");
    c->launches += 2;
  }
  if (row_perm || col_perm) {
    bsvd_status s = read_errors(c, "partition");
    if (s != BSVD_OK) return s;
  }

  const void *du = nullptr, *di = nullptr, *dx = nullptr;
  CK(device_view(c, u, sizeof(int32_t) * nnz, c->s_a, &du), "partition");
  CK(device_view(c, i, sizeof(int32_t) * nnz, c->s_b, &di), "partition");
  CK(device_view(c, x, sizeof(float) * nnz, c->s_c, &dx), "partition");

  CK(cudaMemsetAsync(c->d_counts.p, 0, sizeof(unsigned long long) * nb, c->st),
     "partition");
  CK(cudaMemsetAsync(c->d_sums.p, 0, sizeof(long long) * nb, c->st),
     "partition");
  CK(cudaMemsetAsync(c->d_maxabs.p, 0, sizeof(unsigned int), c->st),
     "partition");
  if (c->w32)
    CK(cudaMemsetAsync(c->d_W.p, 0, sizeof(float) * std::max<int64_t>(off, 1),
                       c->st), "partition");
  const GridDesc g = c->grid();
  std::fill(c->phase_ms, c->phase_ms + 8, 0.0);
  mark(c, 0);
  CK(launch_count(g, nnz, (const int32_t *)du, (const int32_t *)di,
                  (const float *)dx, nb, c->d_counts.as<unsigned long long>(),
                  c->d_sums.as<long long>(), c->d_maxabs.as<unsigned int>(),
                  c->d_err.as<int32_t>(), c->st), "partition: count");
  CK(launch_means(nb, c->d_counts.as<unsigned long long>(),
                  c->d_sums.as<long long>(), c->d_maxabs.as<unsigned int>(),
                  c->d_mu.as<float>(), c->d_err.as<int32_t>(), c->st),
     "partition: means");
  __nv_bfloat16 *wh = nullptr;
  if (c->cfg.precision == BSVD_BF16) {
    CK(c->d_VX.ensure(2 * std::max<int64_t>(vxoff, 1)), "partition");
    CK(cudaMemsetAsync(c->d_VX.p, 0, 2 * std::max<int64_t>(vxoff, 1), c->st),
       "partition");
    wh = c->d_VX.as<__nv_bfloat16>();
  }
  CK(launch_scatter(g, c->d_meta.as<BlockMeta>(), nnz, (const int32_t *)du,
                    (const int32_t *)di, (const float *)dx,
                    c->d_mu.as<float>(), c->w32 ? c->d_W.as<float>() : nullptr,
                    wh, c->st),
     "partition: scatter");
  c->launches += nnz > 0 ? 3 : 1;
  // bf16 planes for the exact tensor-core Gram
  c->tc_planes = c->cfg.gram_path != 1 && c->cfg.precision == BSVD_FP32;
  c->tc_exact = false;
  if (c->tc_planes) {
    CK(c->d_VX.ensure(2 * std::max<int64_t>(vxoff, 1)), "partition");
    CK(c->d_shift.ensure(sizeof(float) * nb), "partition");
    CK(c->d_delta.ensure(sizeof(float) * nb), "partition");
    CK(c->d_flag.ensure(sizeof(int32_t)), "partition");
    CK(cudaMemsetAsync(c->d_VX.p, 0, 2 * std::max<int64_t>(vxoff, 1), c->st),
       "partition");
    CK(cudaMemsetAsync(c->d_flag.p, 0, sizeof(int32_t), c->st), "partition");
    CK(launch_plane_shift(nb, c->d_counts.as<unsigned long long>(),
                          c->d_sums.as<long long>(), c->d_shift.as<float>(),
                          c->d_delta.as<float>(), c->st), "partition: shift");
    CK(launch_scatter_planes(g, c->d_meta.as<BlockMeta>(), nnz,
                             (const int32_t *)du, (const int32_t *)di,
                             (const float *)dx, c->d_shift.as<float>(),
                             c->d_VX.as<__nv_bfloat16>(), c->d_flag.as<int32_t>(),
                             c->st), "partition: planes");
    c->launches += nnz > 0 ? 2 : 1;
  }
  mark(c, 1);
  bsvd_status s = read_errors(c, "partition");
  if (s != BSVD_OK) return s;
  take(c, 0, 0, 1);
  if (c->tc_planes) {
    int32_t flag = 0;
    CK(cudaMemcpyAsync(&flag, c->d_flag.p, sizeof flag, cudaMemcpyDeviceToHost,
                       c->st), "partition");
    CK(cudaStreamSynchronize(c->st), "partition");
    c->tc_exact = (flag & kErrNotExact) == 0;
  }
  if ((c->tc_planes && c->tc_exact) || c->cfg.precision == BSVD_BF16) {
    const int64_t plane_rows = c->cfg.precision == BSVD_BF16 ? 1 : 2;
    {
      // one TMA map per block over its bf16 rows: [Y; M] or the bf16 W
      EncodeTiledFn enc = tensor_map_encoder();
      if (!enc) return fail(c, BSVD_ECUDA, "partition: no cuTensorMapEncodeTiled");
      std::vector<CUtensorMap> maps(nb);
      std::memset(maps.data(), 0, sizeof(CUtensorMap) * nb);
      for (int32_t b = 0; b < nb; ++b) {
        const BlockMeta &bm = c->meta[b];
        if (bm.s == 0 || !bm.owned) continue;
        cuuint64_t dims[2] = {(cuuint64_t)bm.L_pad,
                              (cuuint64_t)(plane_rows * bm.s128)};
        cuuint64_t strides[1] = {(cuuint64_t)bm.L_pad * 2};
        cuuint32_t box[2] = {64, 128};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&maps[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         c->d_VX.as<__nv_bfloat16>() + bm.vx_off, dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          return fail(c, BSVD_ECUDA, "partition: tensor map %d failed (%d)", b,
                      (int)r);
      }
      CK(c->d_maps.ensure(sizeof(CUtensorMap) * nb), "partition");
      // stream-ordered: the context's stream may be a non-blocking one
      CK(cudaMemcpyAsync(c->d_maps.p, maps.data(), sizeof(CUtensorMap) * nb,
                         cudaMemcpyHostToDevice, c->st), "partition");
      CK(cudaStreamSynchronize(c->st), "partition");
    }
  }
  if (c->cfg.precision == BSVD_TF32) {
    // one TMA map per block over its float32 W (s_pad x L_pad)
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return fail(c, BSVD_ECUDA, "partition: no cuTensorMapEncodeTiled");
    std::vector<CUtensorMap> maps(nb);
    std::memset(maps.data(), 0, sizeof(CUtensorMap) * nb);
    for (int32_t b = 0; b < nb; ++b) {
      const BlockMeta &bm = c->meta[b];
      if (bm.s == 0 || !bm.owned) continue;
      cuuint64_t dims[2] = {(cuuint64_t)bm.L_pad, (cuuint64_t)bm.s_pad};
      cuuint64_t strides[1] = {(cuuint64_t)bm.L_pad * 4};
      cuuint32_t box[2] = {32, 128};
      cuuint32_t es[2] = {1, 1};
      CUresult r = enc(&maps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                       c->d_W.as<float>() + bm.w_off, dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(c, BSVD_ECUDA, "partition: tensor map %d failed (%d)", b,
                    (int)r);
    }
    CK(c->d_wmaps.ensure(sizeof(CUtensorMap) * nb), "partition");
    CK(cudaMemcpyAsync(c->d_wmaps.p, maps.data(), sizeof(CUtensorMap) * nb,
                       cudaMemcpyHostToDevice, c->st), "partition");
    CK(cudaStreamSynchronize(c->st), "partition");
  }
  c->parted = true;
  return BSVD_OK;
}

bsvd_status bsvd_partition(bsvd_ctx *c, int64_t m, int64_t n, int64_t nnz,
                           const int32_t *u, const int32_t *i,
                           const float *x, int32_t p, int32_t q,
                           const int64_t *row_bounds,
                           const int64_t *col_bounds,
                           const int32_t *row_perm, const int32_t *col_perm) {
  return partition_impl(c, m, n, nnz, u, i, x, p, q, row_bounds, col_bounds,
                        row_perm, col_perm, false);
}

bsvd_status bsvd_partition_diag(bsvd_ctx *c, int32_t nb,
                                const int64_t *row_bounds,
                                const int64_t *col_bounds, int64_t nnz,
                                const int32_t *u, const int32_t *i,
                                const float *x) {
  if (!c) return BSVD_EINVAL;
  if (nb < 1 || !row_bounds || !col_bounds)
    return fail(c, BSVD_EINVAL, "partition_diag: need nb >= 1 and bounds");
  return partition_impl(c, row_bounds[nb], col_bounds[nb], nnz, u, i, x, nb,
                        nb, row_bounds, col_bounds, nullptr, nullptr, true);
}

// One side of the activity-quantile grid: perm (host or device, size
// entries) and bounds (host, parts + 1).
static bsvd_status quantile_side(bsvd_ctx *c, const char *what, int64_t size,
                                 int64_t nnz, const int32_t *ids,
                                 int32_t parts, int32_t *perm,
                                 int64_t *bounds) {
  const int64_t padded = quantile_cut_padded(size);
  CK(c->d_qcnt.ensure(sizeof(unsigned int) * size), what);
  CK(c->d_qkeys.ensure(sizeof(unsigned long long) * padded), what);
  CK(c->d_qcum.ensure(sizeof(long long) * (size + 1)), what);
  CK(c->d_qbounds.ensure(sizeof(int64_t) * (parts + 1)), what);
  const bool dev_perm = is_device_ptr(perm);
  int32_t *dperm = perm;
  if (!dev_perm) {
    CK(c->d_qperm.ensure(sizeof(int32_t) * size), what);
    dperm = c->d_qperm.as<int32_t>();
  }
  CK(launch_quantile_cut(ids, nnz, size, parts, c->d_qcnt.as<unsigned int>(),
                         c->d_qkeys.as<unsigned long long>(),
                         c->d_qcum.as<long long>(), dperm,
                         c->d_qbounds.as<int64_t>(), c->d_err.as<int32_t>(),
                         &c->launches, c->st), what);
  if (!dev_perm)
    CK(cudaMemcpyAsync(perm, dperm, sizeof(int32_t) * size,
                       cudaMemcpyDeviceToHost, c->st), what);
  CK(cudaMemcpyAsync(bounds, c->d_qbounds.p, sizeof(int64_t) * (parts + 1),
                     cudaMemcpyDeviceToHost, c->st), what);
  return BSVD_OK;
}

bsvd_status bsvd_quantile_grid(bsvd_ctx *c, int64_t m, int64_t n, int64_t nnz,
                               const int32_t *u, const int32_t *i, int32_t p,
                               int32_t q, int32_t *row_perm,
                               int32_t *col_perm, int64_t *row_bounds,
                               int64_t *col_bounds) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX || nnz < 0 ||
      nnz > (int64_t)UINT32_MAX)
    return fail(c, BSVD_EINVAL, "quantile_grid: bad sizes m=%lld n=%lld "
                "nnz=%lld", (long long)m, (long long)n, (long long)nnz);
  if (p < 1 || q < 1 || p > m || q > n)
    return fail(c, BSVD_EINVAL, "quantile_grid: bad grid %d x %d", p, q);
  if ((nnz > 0 && (!u || !i)) || !row_perm || !col_perm || !row_bounds ||
      !col_bounds)
    return fail(c, BSVD_EINVAL, "quantile_grid: null array");
  const void *du = nullptr, *di = nullptr;
  CK(cudaMemsetAsync(c->d_err.p, 0, sizeof(int32_t), c->st), "quantile_grid");
  CK(device_view(c, u, sizeof(int32_t) * nnz, c->s_a, &du), "quantile_grid");
  CK(device_view(c, i, sizeof(int32_t) * nnz, c->s_b, &di), "quantile_grid");
  bsvd_status s = quantile_side(c, "quantile_grid: rows", m, nnz,
                                (const int32_t *)du, p, row_perm, row_bounds);
  if (s != BSVD_OK) return s;
  s = quantile_side(c, "quantile_grid: columns", n, nnz, (const int32_t *)di,
                    q, col_perm, col_bounds);
  if (s != BSVD_OK) return s;
  return read_errors(c, "quantile_grid");
}

bsvd_status bsvd_partition_quantile(bsvd_ctx *c, int64_t m, int64_t n,
                                    int64_t nnz, const int32_t *u,
                                    const int32_t *i, const float *x,
                                    int32_t p, int32_t q, int64_t *row_bounds,
                                    int64_t *col_bounds) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX || nnz < 0 ||
      nnz > (int64_t)UINT32_MAX)
    return fail(c, BSVD_EINVAL, "partition_quantile: bad sizes m=%lld n=%lld "
                "nnz=%lld", (long long)m, (long long)n, (long long)nnz);
  if (p < 1 || q < 1 || p > m || q > n)
    return fail(c, BSVD_EINVAL, "partition_quantile: bad grid %d x %d", p, q);
  if (nnz > 0 && (!u || !i || !x))
    return fail(c, BSVD_EINVAL, "partition_quantile: null rating arrays");
  const char *what = "partition_quantile";
  // x (host) goes up on its own stream, after whatever the caller's stream
  // still has to do with the staging buffer, while u and i go up and the
  // grid is cut on the caller's stream
  const void *du = nullptr, *di = nullptr, *dx = x;
  bool forked = false;
  if (nnz > 0 && !is_device_ptr(x)) {
    if (!c->up)
      CK(cudaStreamCreateWithFlags(&c->up, cudaStreamNonBlocking), what);
    if (!c->ev_up_fork)
      CK(cudaEventCreateWithFlags(&c->ev_up_fork, cudaEventDisableTiming), what);
    if (!c->ev_up_join)
      CK(cudaEventCreateWithFlags(&c->ev_up_join, cudaEventDisableTiming), what);
    CK(c->s_c.ensure(sizeof(float) * nnz), what);
    CK(cudaEventRecord(c->ev_up_fork, c->st), what);
    CK(cudaStreamWaitEvent(c->up, c->ev_up_fork, 0), what);
    CK(cudaMemcpyAsync(c->s_c.p, x, sizeof(float) * nnz, cudaMemcpyHostToDevice,
                       c->up), what);
    CK(cudaEventRecord(c->ev_up_join, c->up), what);
    dx = c->s_c.p;
    forked = true;
  }
  CK(cudaMemsetAsync(c->d_err.p, 0, sizeof(int32_t), c->st), what);
  CK(device_view(c, u, sizeof(int32_t) * nnz, c->s_a, &du), what);
  CK(device_view(c, i, sizeof(int32_t) * nnz, c->s_b, &di), what);
  // the permutations stay on the device (the partition copies them into
  // the context); the bounds come to the host for the block layout
  CK(c->d_qperm.ensure(sizeof(int32_t) * m), what);
  CK(c->d_qperm2.ensure(sizeof(int32_t) * n), what);
  std::vector<int64_t> rb(p + 1), cb(q + 1);
  bsvd_status s = quantile_side(c, "partition_quantile: rows", m, nnz,
                                (const int32_t *)du, p,
                                c->d_qperm.as<int32_t>(), rb.data());
  if (s == BSVD_OK)
    s = quantile_side(c, "partition_quantile: columns", n, nnz,
                      (const int32_t *)di, q, c->d_qperm2.as<int32_t>(),
                      cb.data());
  // the caller's stream takes the upload over in every case, so no later
  // call reuses the staging buffer while it is still being written
  if (forked) CK(cudaStreamWaitEvent(c->st, c->ev_up_join, 0), what);
  if (s != BSVD_OK) return s;
  s = read_errors(c, what);
  if (s != BSVD_OK) return s;
  if (row_bounds) std::copy(rb.begin(), rb.end(), row_bounds);
  if (col_bounds) std::copy(cb.begin(), cb.end(), col_bounds);
  return partition_impl(c, m, n, nnz, (const int32_t *)du, (const int32_t *)di,
                        (const float *)dx, p, q, rb.data(), cb.data(),
                        c->d_qperm.as<int32_t>(), c->d_qperm2.as<int32_t>(),
                        false);
}

static bsvd_status factor_impl(bsvd_ctx *c, int32_t k, const int32_t *ks);


bsvd_status bsvd_factor(bsvd_ctx *c, int32_t k) {
  return factor_impl(c, k, nullptr);
}

bsvd_status bsvd_factor_ks(bsvd_ctx *c, const int32_t *ks) {
  if (!c) return BSVD_EINVAL;
  if (!ks) return fail(c, BSVD_EINVAL, "factor_ks: null k array");
  return factor_impl(c, 0, ks);
}

static bsvd_status factor_impl(bsvd_ctx *c, int32_t k, const int32_t *ks) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->parted) return fail(c, BSVD_ESTATE, "factor: no partition");
  if (ks) {
    k = 0;
    for (int32_t b = 0; b < c->nblocks; ++b) {
      if (ks[b] < 0 || ks[b] > 56)
        return fail(c, BSVD_EINVAL, "factor: k[%d]=%d outside [0, 56]", b, ks[b]);
      k = std::max(k, ks[b]);
    }
  }
  if (k < 0 || k > 56) return fail(c, BSVD_EINVAL, "factor: k=%d outside [0, 56]", k);
  if (c->cfg.precision == BSVD_FP32 && c->cfg.gram_path == 2 &&
      !(c->tc_planes && c->tc_exact))
    return fail(c, BSVD_EINVAL,
                "factor: tensor-core Gram needs ratings that are small integer "
                "offsets from their block's rounded mean");
  c->factored = false;
  c->any_capped = false;
  c->last_graph = 0;
  c->panel_launches = 0;
  c->k = k;
  c->bsub = subspace_width(k, c->cfg.oversample);
  c->kp = (int32_t)std::max<int64_t>(4, round_up(k, 4));
  const int32_t B = c->bsub, kp = c->kp, nb = c->nblocks;

  const bool proj16 = c->cfg.panel_path == 0 && c->cfg.precision == BSVD_BF16;
  const bool g256 = c->cfg.precision == BSVD_BF16 ||
                    c->cfg.precision == BSVD_TF32;
  const int32_t kn = (int32_t)round_up(kp, 16);
  int64_t goff = 0, xoff = 0, fsoff = 0, floff = 0, fboff = 0;
  std::vector<int4> gt;
  std::vector<int2> rt, lt, pt, pj, ch;
  std::vector<SolverState> st0(nb);
  for (int32_t b = 0; b < nb; ++b) {
    BlockMeta &bm = c->meta[b];
    bm.keff = bm.owned ? std::min(ks ? ks[b] : k, bm.s) : 0;
    bm.g_off = goff;
    bm.x_off = xoff;
    bm.fs_off = fsoff;
    bm.fl_off = floff;
    bm.fb_off = fboff;
    if (bm.owned) {          // another shard's block takes no solver storage
      if (proj16 && bm.s > 0) fboff += project_bf16_bform_elems(bm.s_pad, kn);
      goff += (int64_t)bm.s_pad * bm.s_pad;
      xoff += (int64_t)bm.s_pad * B;
      fsoff += (int64_t)bm.s_pad * kp;
      floff += (int64_t)bm.L_pad * kp;
    }
    SolverState &s = st0[b];
    std::memset(&s, 0, sizeof s);
    s.bsub = std::min(B, bm.s);
    s.status = (bm.s == 0 || bm.keff == 0) ? kConverged : kRunning;
    bm.t0 = (int32_t)rt.size();
    bm.nt = 0;
    bm.pt0 = 0;
    bm.npt = 0;
    bm.pj0 = 0;
    bm.npj = 0;
    bm.ch0 = (int32_t)ch.size();
    bm.nch = 0;
    if (bm.s == 0 || !bm.owned) continue;
    // Gram tiles: 256 x 256 for the single-product tensor-core Grams,
    // 128 x 128 for the exact four-product one and the FP32 SIMT one
    const int32_t tsz = g256 ? 256 : 128;
    const int32_t T = (bm.s_pad + tsz - 1) / tsz;
    for (int32_t ti = 0; ti < T; ++ti)
      for (int32_t tj = ti; tj < T; ++tj) gt.push_back(make_int4(b, ti, tj, 0));
    for (int32_t r = 0; r < bm.s_pad; r += 64) rt.push_back(make_int2(b, r));
    bm.nt = (int32_t)rt.size() - bm.t0;
    for (int32_t r = 0; r < bm.s; r += kChunkRows) ch.push_back(make_int2(b, r));
    bm.nch = (int32_t)ch.size() - bm.ch0;
    for (int32_t l = 0; l < bm.L; l += kProjCols) lt.push_back(make_int2(b, l));
  }
  // 128-row tiles of the panel products (over F_s) and of the projection
  // (over F_L), the blocks in decreasing order of s: a tile of either
  // reduces over s, so its cost grows with s. The persistent products claim
  // tiles in table order and the projection's CTAs start in it, so the
  // longest tiles start first and the shortest fill the end of each
  // launch. A block's tiles stay contiguous; ties keep the block order.
  {
    std::vector<int32_t> order(nb);
    for (int32_t b = 0; b < nb; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return c->meta[a].s > c->meta[b].s;
    });
    for (int32_t b : order) {
      BlockMeta &bm = c->meta[b];
      bm.pt0 = (int32_t)pt.size();
      bm.pj0 = (int32_t)pj.size();
      if (bm.s > 0 && bm.owned) {
        for (int32_t r = 0; r < bm.s_pad; r += 128) pt.push_back(make_int2(b, r));
        for (int32_t l = 0; l < bm.L; l += 128) pj.push_back(make_int2(b, l));
      }
      bm.npt = (int32_t)pt.size() - bm.pt0;
      bm.npj = (int32_t)pj.size() - bm.pj0;
    }
  }
  // Gram tiles longest first (a tile's work grows with its block's L):
  // CTAs start in launch order, so the last ones to start are the short
  // tiles and the launch does not end on one long tile. Each tile writes
  // its own part of G, so the order changes nothing in the result.
  std::stable_sort(gt.begin(), gt.end(), [&](const int4 &x, const int4 &y) {
    return c->meta[x.x].L_pad > c->meta[y.x].L_pad;
  });
  c->n_gtiles = (int32_t)gt.size();
  c->n_rowtiles = (int32_t)rt.size();
  c->n_ltiles = (int32_t)lt.size();
  c->n_ptiles = (int32_t)pt.size();
  c->n_pjtiles = (int32_t)pj.size();
  c->n_chunks = (int32_t)ch.size();
  const bool panel_tc = c->cfg.panel_path == 0;

  CK(c->d_G.ensure(sizeof(float) * std::max<int64_t>(goff, 1)), "factor");
  CK(c->d_X.ensure(sizeof(float) * std::max<int64_t>(xoff, 1)), "factor");
  CK(c->d_Z.ensure(sizeof(float) * std::max<int64_t>(xoff, 1)), "factor");
  CK(c->d_SH.ensure(sizeof(float) * 2 * B * B * std::max<int64_t>(ch.size(), 1)), "factor");
  CK(c->d_chunks.ensure(sizeof(int2) * std::max<size_t>(ch.size(), 1)), "factor");
  CK(c->d_RP.ensure(sizeof(double) * 2 * B * std::max<int64_t>(rt.size(), 1)), "factor");
  CK(c->d_T.ensure(sizeof(float) * B * B * (int64_t)nb), "factor");
  CK(c->d_theta.ensure(sizeof(float) * B * (int64_t)nb), "factor");
  CK(c->d_finv.ensure(sizeof(float) * B * (int64_t)nb), "factor");
  CK(c->d_state.ensure(sizeof(SolverState) * nb), "factor");
  CK(c->d_Fs.ensure(sizeof(float) * std::max<int64_t>(fsoff, 1)), "factor");
  CK(c->d_FL.ensure(sizeof(float) * std::max<int64_t>(floff, 1)), "factor");
  CK(c->d_sigma.ensure(sizeof(double) * kp * (int64_t)nb), "factor");
  CK(c->d_running.ensure(2 * sizeof(int32_t)), "factor");
  CK(c->d_gtiles.ensure(sizeof(int4) * std::max<size_t>(gt.size(), 1)), "factor");
  CK(c->d_rowtiles.ensure(sizeof(int2) * std::max<size_t>(rt.size(), 1)), "factor");
  CK(c->d_ltiles.ensure(sizeof(int2) * std::max<size_t>(lt.size(), 1)), "factor");
  CK(c->d_state0.ensure(sizeof(SolverState) * std::max(nb, 1)), "factor");
  // 128-row tiles of F_s (panel products, finalisation) and of F_L
  // (projection, finalisation), and the finalisation's partials and flips
  CK(c->d_ptiles.ensure(sizeof(int2) * std::max<size_t>(pt.size(), 1)), "factor");
  CK(c->d_pjtiles.ensure(sizeof(int2) * std::max<size_t>(pj.size(), 1)),
     "factor");
  CK(c->d_lpart.ensure(sizeof(ColPartial) * kp *
                       std::max<size_t>(pj.size(), 1)), "factor");
  CK(c->d_spart.ensure(sizeof(ColPartial) * kp *
                       std::max<size_t>(pt.size(), 1)), "factor");
  CK(c->d_flip.ensure((size_t)kp * std::max(nb, 1)), "factor");
  CK(c->d_pctl.ensure(2 * sizeof(int32_t)), "factor");
  CK(cudaMemsetAsync(c->d_pctl.p, 0, 2 * sizeof(int32_t), c->st), "factor");
  CK(c->d_ptime.ensure(3 * sizeof(unsigned long long)), "factor");
  CK(c->d_loopctl.ensure(2 * sizeof(int32_t)), "factor");
  const bool tc_maps = panel_tc && !pt.empty();
  if (tc_maps) {
    CK(c->d_gmaps.ensure(sizeof(CUtensorMap) * nb), "factor");
    CK(c->d_XB.ensure(sizeof(float) * 2 * std::max<int64_t>(xoff, 1)), "factor");
    CK(c->d_ZB.ensure(sizeof(float) * 2 * std::max<int64_t>(xoff, 1)), "factor");
    CK(c->d_xmaps.ensure(sizeof(CUtensorMap) * 2 * nb), "factor");
    CK(c->d_pwmaps.ensure(sizeof(CUtensorMap) * std::max(nb, 1)), "factor");
    if (proj16) {
      CK(c->d_pbmaps.ensure(sizeof(CUtensorMap) * std::max(nb, 1)), "factor");
      CK(c->d_fbmaps.ensure(sizeof(CUtensorMap) * std::max(nb, 1)), "factor");
      CK(c->d_FB.ensure(2 * std::max<int64_t>(fboff, 1)), "factor");
    }
  }
  // The tile tables, the TMA maps and the initial solver state depend only
  // on the block layout (the metadata computed above, which includes every
  // offset and keff), on B, kp and the panel path, and on the device
  // addresses the maps point into. Repeated factorisations of one layout
  // (the usual case: a new partition of the same shape) skip rebuilding
  // and uploading them; uploads from pageable memory would each wait for
  // the stream, and encoding the maps is host work the GPU idles through.
  std::vector<unsigned char> sig;
  {
    auto put = [&](const void *p, size_t n) {
      const unsigned char *b = static_cast<const unsigned char *>(p);
      sig.insert(sig.end(), b, b + n);
    };
    put(c->meta.data(), sizeof(BlockMeta) * nb);
    const int64_t head[4] = {B, kp, panel_tc ? 1 : 0, nb};
    put(head, sizeof head);
    const void *ptrs[] = {c->d_G.p, c->d_W.p, c->d_XB.p, c->d_ZB.p,
                          c->d_gtiles.p, c->d_rowtiles.p, c->d_ltiles.p,
                          c->d_gmaps.p, c->d_xmaps.p, c->d_ptiles.p,
                          c->d_pwmaps.p, c->d_pjtiles.p, c->d_state0.p,
                          c->d_VX.p, c->d_pbmaps.p, c->d_fbmaps.p, c->d_FB.p,
                          c->d_lpart.p, c->d_spart.p, c->d_flip.p,
                          c->d_chunks.p};
    put(ptrs, sizeof ptrs);
  }
  const bool same_layout = sig == c->fsig;
  c->fsig.clear();       // set again once everything below is uploaded

  CK(cudaMemcpyAsync(c->d_meta.p, c->meta.data(), sizeof(BlockMeta) * nb,
                     cudaMemcpyHostToDevice, c->st), "factor");
  if (!same_layout) {
    CK(cudaMemcpyAsync(c->d_state0.p, st0.data(), sizeof(SolverState) * nb,
                       cudaMemcpyHostToDevice, c->st), "factor");
    if (!gt.empty())
      CK(cudaMemcpyAsync(c->d_gtiles.p, gt.data(), sizeof(int4) * gt.size(),
                         cudaMemcpyHostToDevice, c->st), "factor");
    if (!rt.empty())
      CK(cudaMemcpyAsync(c->d_rowtiles.p, rt.data(), sizeof(int2) * rt.size(),
                         cudaMemcpyHostToDevice, c->st), "factor");
    if (!lt.empty())
      CK(cudaMemcpyAsync(c->d_ltiles.p, lt.data(), sizeof(int2) * lt.size(),
                         cudaMemcpyHostToDevice, c->st), "factor");
    if (!pt.empty())
      CK(cudaMemcpyAsync(c->d_ptiles.p, pt.data(), sizeof(int2) * pt.size(),
                         cudaMemcpyHostToDevice, c->st), "factor");
    if (!pj.empty())
      CK(cudaMemcpyAsync(c->d_pjtiles.p, pj.data(), sizeof(int2) * pj.size(),
                         cudaMemcpyHostToDevice, c->st), "factor");
    if (!ch.empty())
      CK(cudaMemcpyAsync(c->d_chunks.p, ch.data(), sizeof(int2) * ch.size(),
                         cudaMemcpyHostToDevice, c->st), "factor");
  }
  if (nb > 0)
    CK(cudaMemcpyAsync(c->d_state.p, c->d_state0.p, sizeof(SolverState) * nb,
                       cudaMemcpyDeviceToDevice, c->st), "factor");
  if (tc_maps && !same_layout) {
    // one TMA map per block over its Gram matrix (s_pad x s_pad float32,
    // 128-row x 32-float boxes) for the tensor-core panel products
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return fail(c, BSVD_ECUDA, "factor: no cuTensorMapEncodeTiled");
    c->h_gmaps.assign(nb, CUtensorMap());
    std::memset(c->h_gmaps.data(), 0, sizeof(CUtensorMap) * nb);
    for (int32_t b = 0; b < nb; ++b) {
      const BlockMeta &bm = c->meta[b];
      if (bm.s == 0 || !bm.owned) continue;
      cuuint64_t dims[2] = {(cuuint64_t)bm.s_pad, (cuuint64_t)bm.s_pad};
      cuuint64_t strides[1] = {(cuuint64_t)bm.s_pad * 4};
      cuuint32_t box[2] = {32, 128};
      cuuint32_t es[2] = {1, 1};
      CUresult r = enc(&c->h_gmaps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                       c->d_G.as<float>() + bm.g_off, dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(c, BSVD_ECUDA, "factor: Gram tensor map %d failed (%d)", b,
                    (int)r);
    }
    CK(c->d_gmaps.ensure(sizeof(CUtensorMap) * nb), "factor");
    CK(cudaMemcpyAsync(c->d_gmaps.p, c->h_gmaps.data(),
                       sizeof(CUtensorMap) * nb, cudaMemcpyHostToDevice, c->st),
       "factor");
    // and over the B forms of the two panel buffers (per block: s_pad / 32
    // chunks of 2 B rows x 32 floats, one chunk per box, 128-byte swizzle):
    // maps [0, nb) read X, maps [nb, 2 nb) read Z
    CK(c->d_XB.ensure(sizeof(float) * 2 * std::max<int64_t>(xoff, 1)), "factor");
    CK(c->d_ZB.ensure(sizeof(float) * 2 * std::max<int64_t>(xoff, 1)), "factor");
    c->h_xmaps.assign(2 * (size_t)nb, CUtensorMap());
    std::memset(c->h_xmaps.data(), 0, sizeof(CUtensorMap) * 2 * nb);
    for (int h = 0; h < 2; ++h) {
      float *bform = h == 0 ? c->d_XB.as<float>() : c->d_ZB.as<float>();
      for (int32_t b = 0; b < nb; ++b) {
        const BlockMeta &bm = c->meta[b];
        if (bm.s == 0 || !bm.owned) continue;
        cuuint64_t dims[2] = {32, (cuuint64_t)(bm.s_pad / 32) * 2 * B};
        cuuint64_t strides[1] = {128};
        cuuint32_t box[2] = {32, (cuuint32_t)(2 * B)};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&c->h_xmaps[(size_t)h * nb + b],
                         CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, bform + 2 * bm.x_off,
                         dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          return fail(c, BSVD_ECUDA, "factor: panel tensor map %d failed (%d)",
                      b, (int)r);
      }
    }
    CK(c->d_xmaps.ensure(sizeof(CUtensorMap) * 2 * nb), "factor");
    CK(cudaMemcpyAsync(c->d_xmaps.p, c->h_xmaps.data(),
                       sizeof(CUtensorMap) * 2 * nb, cudaMemcpyHostToDevice,
                       c->st), "factor");
    // the tensor-core projection F_L = W^T F_s: one TMA map per block over
    // W (s_pad rows x L_pad columns, float32, boxes of 32 rows x 128
    // columns, plain layout) and 128-column tiles
    c->h_pwmaps.assign(nb, CUtensorMap());
    std::memset(c->h_pwmaps.data(), 0, sizeof(CUtensorMap) * nb);
    for (int32_t b = 0; b < nb && !proj16; ++b) {
      const BlockMeta &bm = c->meta[b];
      if (bm.s == 0 || bm.L == 0 || !bm.owned) continue;
      cuuint64_t dims[2] = {(cuuint64_t)bm.L_pad, (cuuint64_t)bm.s_pad};
      cuuint64_t strides[1] = {(cuuint64_t)bm.L_pad * 4};
      cuuint32_t box[2] = {128, 32};
      cuuint32_t es[2] = {1, 1};
      CUresult r = enc(&c->h_pwmaps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                       c->d_W.as<float>() + bm.w_off, dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(c, BSVD_ECUDA, "factor: W tensor map %d failed (%d)", b,
                    (int)r);
    }
    CK(c->d_pwmaps.ensure(sizeof(CUtensorMap) * std::max(nb, 1)), "factor");
    CK(cudaMemcpyAsync(c->d_pwmaps.p, c->h_pwmaps.data(),
                       sizeof(CUtensorMap) * nb, cudaMemcpyHostToDevice,
                       c->st), "factor");
    if (proj16) {
      // the BF16 form's projection: maps over the bf16 blocks (s128 rows x
      // L_pad, boxes of 64 rows x 128 columns, plain layout) and over F_s's
      // bf16 B form (rows of 64 values, 2 kn-row boxes, 128-byte swizzle)
      c->h_pbmaps.assign(nb, CUtensorMap());
      c->h_fbmaps.assign(nb, CUtensorMap());
      std::memset(c->h_pbmaps.data(), 0, sizeof(CUtensorMap) * nb);
      std::memset(c->h_fbmaps.data(), 0, sizeof(CUtensorMap) * nb);
      for (int32_t b = 0; b < nb; ++b) {
        const BlockMeta &bm = c->meta[b];
        if (bm.s == 0 || bm.L == 0 || !bm.owned) continue;
        cuuint64_t dims[2] = {(cuuint64_t)bm.L_pad, (cuuint64_t)bm.s128};
        cuuint64_t strides[1] = {(cuuint64_t)bm.L_pad * 2};
        cuuint32_t box[2] = {128, 64};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&c->h_pbmaps[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         c->d_VX.as<__nv_bfloat16>() + bm.vx_off, dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          return fail(c, BSVD_ECUDA, "factor: bf16 W tensor map %d failed (%d)",
                      b, (int)r);
        const int64_t rows = project_bf16_bform_elems(bm.s_pad, kn) / 64;
        cuuint64_t fdims[2] = {64, (cuuint64_t)rows};
        cuuint64_t fstrides[1] = {128};
        cuuint32_t fbox[2] = {64, (cuuint32_t)(2 * kn)};
        r = enc(&c->h_fbmaps[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                c->d_FB.as<__nv_bfloat16>() + bm.fb_off, fdims, fstrides, fbox,
                es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          return fail(c, BSVD_ECUDA, "factor: F_s bf16 tensor map %d failed (%d)",
                      b, (int)r);
      }
      CK(cudaMemcpyAsync(c->d_pbmaps.p, c->h_pbmaps.data(),
                         sizeof(CUtensorMap) * nb, cudaMemcpyHostToDevice,
                         c->st), "factor");
      CK(cudaMemcpyAsync(c->d_fbmaps.p, c->h_fbmaps.data(),
                         sizeof(CUtensorMap) * nb, cudaMemcpyHostToDevice,
                         c->st), "factor");
    }
  }
  c->fsig = std::move(sig);
  CK(cudaMemsetAsync(c->d_Fs.p, 0, sizeof(float) * std::max<int64_t>(fsoff, 1), c->st), "factor");
  CK(cudaMemsetAsync(c->d_FL.p, 0, sizeof(float) * std::max<int64_t>(floff, 1), c->st), "factor");
  CK(cudaMemsetAsync(c->d_sigma.p, 0, sizeof(double) * kp * (int64_t)nb, c->st), "factor");

  if (k > 0) {
    EigBuffers e;
    e.meta = c->d_meta.as<BlockMeta>();
    e.state = c->d_state.as<SolverState>();
    e.G = c->d_G.as<float>();
    e.X = c->d_X.as<float>();
    e.Z = c->d_Z.as<float>();
    e.SH = c->d_SH.as<float>();
    e.RP = c->d_RP.as<double>();
    e.T = c->d_T.as<float>();
    e.theta = c->d_theta.as<float>();
    e.Fs = c->d_Fs.as<float>();
    e.Finv = c->d_finv.as<float>();
    e.running = c->d_running.as<int32_t>();
    // k_rotate keeps X's B form current for the tensor-core products
    e.XB = panel_tc ? c->d_XB.as<float>() : nullptr;
    e.bsub = B; e.kp = kp; e.k = k; e.nblocks = nb;
    e.nsm = c->nsm;
    e.max_iters = c->cfg.max_iters;
    e.max_sweeps = c->cfg.max_sweeps;
    e.max_degree = c->cfg.cheb_degree;
    e.tol = (float)c->cfg.tol;
    e.seed = c->cfg.seed;
    const int2 *rtd = c->d_rowtiles.as<int2>();
    const int nrt = c->n_rowtiles;
    // out = alpha G in + beta in + gamma in2 (see launch_gpanel). The
    // tensor-core path reads the B form of `in` and writes that of `out`.
    auto panel = [&](int mode, int step, int deg, const float *in,
                     const float *in2, float *out) -> cudaError_t {
      if (panel_tc) {
        const CUtensorMap *xm = c->d_xmaps.as<CUtensorMap>() +
                                (in == e.X ? 0 : (size_t)nb);
        float *out_bf = out == e.X ? c->d_XB.as<float>() : c->d_ZB.as<float>();
        return launch_gpanel_tc(B, e.meta, e.state, c->d_ptiles.as<int2>(),
                                c->n_ptiles, c->nsm, c->d_pctl.as<int32_t>(),
                                c->d_ptime.as<unsigned long long>(),
                                c->d_gmaps.as<CUtensorMap>(), xm, in, in2, out,
                                out_bf, mode, step, c->d_err.as<int32_t>(),
                                c->st);
      }
      return launch_gpanel(e, rtd, nrt, mode, step, deg, in, in2, out, c->st);
    };
    // B form of X after the random start (k_rotate writes it afterwards)
    auto bform_x = [&]() -> cudaError_t {
      if (!panel_tc) return cudaSuccess;
      ++c->launches;
      return launch_bform(B, e.meta, e.state, c->d_ptiles.as<int2>(),
                          c->n_ptiles, e.X, c->d_XB.as<float>(), c->st);
    };

    std::fill(c->phase_ms + 1, c->phase_ms + 4, 0.0);
    std::fill(c->phase_ms + 5, c->phase_ms + 8, 0.0);
    c->gram_used = c->cfg.precision == BSVD_TF32   ? 3
                   : c->cfg.precision == BSVD_BF16 ? 4
                   : (c->tc_planes && c->tc_exact) ? 2
                                                   : 1;
    // The device work of one factorisation, in four parts: the Gram, the
    // start basis and its first product (pre); one Rayleigh-Ritz step (rr);
    // one Chebyshev filter of degree deg and the product that follows it
    // (filter); the projection and the finalisation (post). Each returns
    // the first error and counts its kernels in c->launches.
    auto pre = [&]() -> cudaError_t {
      cudaError_t r = cudaSuccess;
      mark(c, 0);
      if (c->gram_used == 4)
        r = launch_gram_bf16(c->d_meta.as<BlockMeta>(), c->d_gtiles.as<int4>(),
                             c->n_gtiles, c->d_maps.as<CUtensorMap>(), e.G,
                             c->d_err.as<int32_t>(), c->st);
      else if (c->gram_used == 3)
        r = launch_gram_tf32(c->d_meta.as<BlockMeta>(), c->d_gtiles.as<int4>(),
                             c->n_gtiles, c->d_wmaps.as<CUtensorMap>(), e.G,
                             c->d_err.as<int32_t>(), c->st);
      else if (c->gram_used == 2)
        r = launch_gram_tc(c->d_meta.as<BlockMeta>(), c->d_gtiles.as<int4>(),
                           c->n_gtiles, c->d_maps.as<CUtensorMap>(),
                           c->d_delta.as<float>(), e.G, c->d_err.as<int32_t>(),
                           c->st);
      else
        r = launch_gram_f32(c->d_meta.as<BlockMeta>(), c->d_gtiles.as<int4>(),
                            c->n_gtiles, c->d_W.as<float>(), e.G, c->st);
      if (r != cudaSuccess) return r;
      mark(c, 1);
      if ((r = launch_init_panels(e, rtd, nrt, c->st)) != cudaSuccess) return r;
      if ((r = bform_x()) != cudaSuccess) return r;
      if ((r = panel(0, 0, 0, e.X, nullptr, e.Z)) != cudaSuccess) return r;
      c->launches += (c->n_gtiles > 0) + 2 * (nrt > 0);
      return cudaSuccess;
    };
    auto rr = [&]() -> cudaError_t {
      cudaError_t r;
      if ((r = launch_small_gram(e, c->d_chunks.as<int2>(), c->n_chunks,
                                 c->st)) != cudaSuccess)
        return r;
      if ((r = launch_rr_solve(e, c->st)) != cudaSuccess) return r;
      if ((r = launch_rotate(e, rtd, nrt, c->st)) != cudaSuccess) return r;
      // k_rotate clears the running counters that k_check fills
      if (nrt == 0 &&
          (r = cudaMemsetAsync(e.running, 0, 2 * sizeof(int32_t), c->st)) !=
              cudaSuccess)
        return r;
      if ((r = launch_check(e, c->st)) != cudaSuccess) return r;
      c->launches += 2 + 2 * (nrt > 0);
      return cudaSuccess;
    };
    // Chebyshev filter of even degree: Y_1 -> Z, Y_2 -> X, ..., Y_d -> X;
    // step j reads Y_{j-1}, Y_{j-2} and overwrites Y_{j-2} with Y_j. A block
    // whose own degree is lower skips the later steps, so its Y_d is in X.
    auto fstep = [&](int j) -> cudaError_t {
      const bool even = j % 2 == 0;
      const float *in = even ? e.Z : e.X;
      const float *in2 = j == 1 ? nullptr : (even ? e.X : e.Z);
      float *out = even ? e.X : e.Z;
      c->launches += (nrt > 0);
      return panel(j == 1 ? 1 : 2, j, 0, in, in2, out);
    };
    auto fprod = [&]() -> cudaError_t {
      c->launches += (nrt > 0);
      return panel(0, 0, 0, e.X, nullptr, e.Z);
    };
    auto filter = [&](int deg) -> cudaError_t {
      cudaError_t r;
      for (int j = 1; j <= deg; ++j)
        if ((r = fstep(j)) != cudaSuccess) return r;
      return fprod();
    };
    auto post = [&]() -> cudaError_t {
      cudaError_t r;
      mark(c, 2);
      if ((r = launch_publish_fs(e, c->d_ptiles.as<int2>(), c->n_ptiles,
                                 c->st)) != cudaSuccess)
        return r;
      c->launches += (c->n_ptiles > 0);
      if (proj16) {
        // F_L from the bf16 blocks, F_s split into bf16 hi and lo
        if ((r = launch_bform_fs16(e.meta, c->d_ptiles.as<int2>(), c->n_ptiles,
                                   e.Fs, kp, kn, c->d_FB.as<__nv_bfloat16>(),
                                   c->st)) != cudaSuccess)
          return r;
        if ((r = launch_project_bf16(e.meta, c->d_pjtiles.as<int2>(),
                                     c->n_pjtiles, c->d_pbmaps.as<CUtensorMap>(),
                                     c->d_fbmaps.as<CUtensorMap>(),
                                     c->d_FL.as<float>(), kp, kn,
                                     c->d_err.as<int32_t>(), c->st)) !=
            cudaSuccess)
          return r;
        c->launches += (c->n_ptiles > 0);
      } else if (panel_tc) {
        // F_s's split form goes into X's B-form buffer, free after the loop,
        // and is read through X's maps
        if ((r = launch_bform_fs(B, e.meta, c->d_ptiles.as<int2>(),
                                 c->n_ptiles, e.Fs, kp, c->d_XB.as<float>(),
                                 c->st)) != cudaSuccess)
          return r;
        if ((r = launch_project_tc(B, e.meta, c->d_pjtiles.as<int2>(),
                                   c->n_pjtiles, c->d_pwmaps.as<CUtensorMap>(),
                                   c->d_xmaps.as<CUtensorMap>(),
                                   c->d_FL.as<float>(), kp,
                                   c->d_err.as<int32_t>(), c->st)) !=
            cudaSuccess)
          return r;
        c->launches += (c->n_ptiles > 0);
      } else {
        if ((r = launch_project(c->d_meta.as<BlockMeta>(),
                                c->d_ltiles.as<int2>(), c->n_ltiles,
                                c->d_W.as<float>(), e.Fs, c->d_FL.as<float>(),
                                kp, c->st)) != cudaSuccess)
          return r;
      }
      if ((r = launch_finalize(c->d_meta.as<BlockMeta>(), nb,
                               c->d_pjtiles.as<int2>(), c->n_pjtiles,
                               c->d_ptiles.as<int2>(), c->n_ptiles, e.Fs,
                               c->d_FL.as<float>(), c->d_sigma.as<double>(), kp,
                               c->d_lpart.as<ColPartial>(),
                               c->d_spart.as<ColPartial>(),
                               c->d_flip.as<unsigned char>(), &c->launches,
                               c->st)) != cudaSuccess)
        return r;
      c->launches += (c->n_ltiles > 0);
      mark(c, 3);
      return cudaSuccess;
    };

    // Device-driven form: the same kernels captured once per layout into a
    // CUDA graph whose eigen loop is a conditional WHILE node; k_loopctl
    // decides on the device whether another step runs, so no step waits on
    // the host. The first factorisation of a layout runs the host-driven
    // loop below (a layout seen once may never repeat, and capturing costs
    // about as much as a run); from the second on, the graph.
    {
      std::vector<unsigned char> key = c->fsig;
      const int64_t extra[4] = {c->gram_used, k, B, kp};
      const unsigned char *eb = reinterpret_cast<const unsigned char *>(extra);
      key.insert(key.end(), eb, eb + sizeof extra);
      const void *bufs[] = {c->d_meta.p, c->d_state.p, c->d_G.p, c->d_X.p,
                            c->d_Z.p, c->d_SH.p, c->d_RP.p, c->d_T.p,
                            c->d_theta.p, c->d_Fs.p, c->d_FL.p, c->d_sigma.p,
                            c->d_running.p, c->d_err.p, c->d_maps.p,
                            c->d_delta.p, c->d_wmaps.p, c->d_pctl.p,
                            c->d_ptime.p, c->d_loopctl.p, c->d_finv.p};
      const unsigned char *pb = reinterpret_cast<const unsigned char *>(bufs);
      key.insert(key.end(), pb, pb + sizeof bufs);
      c->gkey_now.swap(key);
    }
    const bool key_seen = c->gkey_now == c->gkey_prev;
    const int loop = c->cfg.loop;
    const bool want_graph = loop == 2 || (loop == 0 && key_seen);
    bool ran_graph = false;
    if (want_graph && !c->graph_failed) {
      if (!c->gexec || c->gkey_now != c->gkey_exec) {
        if (c->gexec) {
          cudaGraphExecDestroy(c->gexec);
          c->gexec = nullptr;
        }
        c->graph_err.clear();
        if (build_graph(c, pre, rr, fstep, fprod, post) != cudaSuccess) {
          cudaGetLastError();
          c->graph_failed = true;     // keep to the host-driven loop
          if (loop == 2)
            return fail(c, BSVD_ECUDA, "factor: the eigen loop's graph could "
                        "not be built (%s)", c->graph_err.c_str());
        } else {
          c->gkey_exec = c->gkey_now;
        }
      }
      if (c->gexec) {
        CK(reset_ptime(c), "factor");
        CK(cudaGraphLaunch(c->gexec, c->st), "factor: graph");
        c->launches += c->graph_static_launches;
        ran_graph = true;
      }
    }
    if (!ran_graph) {
      CK(reset_ptime(c), "factor");
      CK(pre(), "factor: Gram and start");
      for (int it = 0; it <= c->cfg.max_iters + 1; ++it) {
        mark(c, 6);
        CK(rr(), "factor: Rayleigh-Ritz");
        mark(c, 7);
        // The counters reach the host through mapped pinned memory, written
        // by k_publish; this thread polls the sequence word. That avoids a
        // copy and a stream synchronisation per step. If the word does not
        // arrive within kPollMs (an error, or a very slow step), the stream
        // synchronisation below waits and reports any error.
        if (!c->h_run) {
          CK(cudaHostAlloc(&c->h_run, 4 * sizeof(int32_t), cudaHostAllocMapped),
             "factor");
          c->h_run[2] = 0;
          CK(cudaHostGetDevicePointer(&c->d_run_host, c->h_run, 0), "factor");
        }
        const int32_t seq = ++c->run_seq;
        CK(launch_publish(e.running, c->d_run_host, seq, c->st),
           "factor: publish");
        ++c->launches;
        {
          volatile int32_t *hr = c->h_run;
          const auto t0 = std::chrono::steady_clock::now();
          bool seen = false;
          for (uint32_t spin = 0;; ++spin) {
            if (hr[2] == seq) { seen = true; break; }
            if ((spin & 1023u) == 0 &&
                std::chrono::steady_clock::now() - t0 >
                    std::chrono::milliseconds(kPollMs))
              break;
          }
          if (!seen) CK(cudaStreamSynchronize(c->st), "factor");
          std::atomic_thread_fence(std::memory_order_acquire);
        }
        const int32_t run_deg[2] = {c->h_run[0], c->h_run[1]};
        if (c->cfg.profile) {
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]) == cudaSuccess)
            c->phase_ms[6] += ms;
          cudaGetLastError();
        }
        if (run_deg[0] == 0) break;
        CK(filter(std::min(c->cfg.cheb_degree, std::max(2, run_deg[1]))),
           "factor: filter");
      }
      CK(post(), "factor: projection");
    }
    c->gkey_prev = c->gkey_now;
    std::vector<SolverState> fin(nb);
    CK(cudaMemcpyAsync(fin.data(), c->d_state.p, sizeof(SolverState) * nb,
                       cudaMemcpyDeviceToHost, c->st), "factor");
    CK(cudaStreamSynchronize(c->st), "factor");
    for (int32_t b = 0; b < nb; ++b)
      if (fin[b].status != kConverged) c->any_capped = true;
    take(c, 1, 0, 1);
    take(c, 2, 1, 2);
    take(c, 3, 2, 3);
    {
      // the panel products' own time (summed over launches on the device),
      // and in graph form the loop's kernel count
      unsigned long long pt[3] = {0, 0, 0};
      int32_t loops[2] = {0, 0};
      CK(cudaMemcpyAsync(pt, c->d_ptime.p, sizeof pt, cudaMemcpyDeviceToHost,
                         c->st), "factor");
      if (ran_graph)
        CK(cudaMemcpyAsync(loops, c->d_loopctl.p, sizeof loops,
                           cudaMemcpyDeviceToHost, c->st), "factor");
      CK(cudaStreamSynchronize(c->st), "factor");
      c->phase_ms[5] = (double)pt[0] * 1e-6;
      c->panel_launches = (int64_t)pt[2];
      // loop steps times their unconditional kernels, plus the filter
      // steps the loop control opened
      if (ran_graph)
        c->launches += (int64_t)loops[0] * c->graph_loop_launches +
                       (int64_t)loops[1] * (c->n_rowtiles > 0 ? 1 : 0);
      c->last_graph = ran_graph ? 2 : 1;
    }
    // in graph form the Rayleigh-Ritz kernels are not timed on their own:
    // what the eigen phase spends outside the products
    if (ran_graph) c->phase_ms[6] = std::max(0.0, c->phase_ms[2] - c->phase_ms[5]);
    c->phase_ms[7] = std::max(0.0, c->phase_ms[2] - c->phase_ms[5] - c->phase_ms[6]);
  }
  CK(cudaStreamSynchronize(c->st), "factor");
  {
    bsvd_status es = read_errors(c, "factor");
    if (es != BSVD_OK) return es;
  }
  c->factored = true;
  if (c->any_capped)
    return fail(c, BSVD_ENOTCONV, "factor: some blocks hit the iteration cap");
  return BSVD_OK;
}

static PredictArgs predict_args(bsvd_ctx *c) {
  PredictArgs a;
  a.g = c->grid();
  a.meta = c->d_meta.as<BlockMeta>();
  a.mu = c->d_mu.as<float>();
  a.Fs = c->d_Fs.as<float>();
  a.FL = c->d_FL.as<float>();
  a.kp = c->kp;
  a.clamp = c->cfg.clamp;
  a.lo = c->cfg.clamp_lo;
  a.hi = c->cfg.clamp_hi;
  return a;
}

bsvd_status bsvd_predict(bsvd_ctx *c, int64_t nq, const int32_t *u,
                         const int32_t *i, float *yhat) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->factored) return fail(c, BSVD_ESTATE, "predict: no factors");
  if (nq < 0 || (nq > 0 && (!u || !i || !yhat)))
    return fail(c, BSVD_EINVAL, "predict: bad arguments");
  if (nq == 0) return BSVD_OK;
  const void *du, *di;
  CK(device_view(c, u, sizeof(int32_t) * nq, c->s_a, &du), "predict");
  CK(device_view(c, i, sizeof(int32_t) * nq, c->s_b, &di), "predict");
  const bool dev_out = is_device_ptr(yhat);
  float *out = yhat;
  if (!dev_out) {
    CK(c->s_out.ensure(sizeof(float) * nq), "predict");
    out = c->s_out.as<float>();
  }
  mark(c, 4);
  CK(launch_predict(predict_args(c), nq, (const int32_t *)du,
                    (const int32_t *)di, out, c->d_err.as<int32_t>(), c->st),
     "predict");
  mark(c, 5);
  c->launches += 1;
  if (!dev_out)
    CK(cudaMemcpyAsync(yhat, out, sizeof(float) * nq, cudaMemcpyDeviceToHost,
                       c->st), "predict");
  bsvd_status s = read_errors(c, "predict");
  if (s == BSVD_OK) take(c, 4, 4, 5);
  return s;
}

bsvd_status bsvd_rmse(bsvd_ctx *c, int64_t nq, const int32_t *u,
                      const int32_t *i, const float *y, double *out_rmse) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->factored) return fail(c, BSVD_ESTATE, "rmse: no factors");
  if (nq < 1 || !u || !i || !y || !out_rmse)
    return fail(c, BSVD_EINVAL, "rmse: bad arguments");
  const void *du, *di, *dy;
  CK(device_view(c, u, sizeof(int32_t) * nq, c->s_a, &du), "rmse");
  CK(device_view(c, i, sizeof(int32_t) * nq, c->s_b, &di), "rmse");
  CK(device_view(c, y, sizeof(float) * nq, c->s_c, &dy), "rmse");
  CK(c->d_partials.ensure(sizeof(double) * 2 * kSqerrBlocks), "rmse");
  CK(c->d_rmse.ensure(2 * sizeof(double)), "rmse");
  mark(c, 4);
  CK(launch_sqerr(predict_args(c), nq, (const int32_t *)du,
                  (const int32_t *)di, (const float *)dy,
                  c->d_partials.as<double>(), c->d_rmse.as<double>(),
                  c->d_err.as<int32_t>(), c->st), "rmse");
  mark(c, 5);
  c->launches += 2;
  double sum = 0;
  CK(cudaMemcpyAsync(&sum, c->d_rmse.p, sizeof sum, cudaMemcpyDeviceToHost,
                     c->st), "rmse");
  bsvd_status s = read_errors(c, "rmse");
  if (s != BSVD_OK) return s;
  take(c, 4, 4, 5);
  *out_rmse = std::sqrt(sum / (double)nq);
  return BSVD_OK;
}

bsvd_status bsvd_set_owned(bsvd_ctx *c, int32_t nblocks,
                           const uint8_t *owned) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (nblocks < 0 || (nblocks > 0 && !owned))
    return fail(c, BSVD_EINVAL, "set_owned: bad arguments");
  c->own.assign(owned, owned + nblocks);
  for (uint8_t &v : c->own) v = v ? 1 : 0;
  c->parted = false;         // the next partition lays out the owned blocks
  c->factored = false;
  return BSVD_OK;
}

bsvd_status bsvd_sqerr(bsvd_ctx *c, int64_t nq, const int32_t *u,
                       const int32_t *i, const float *y, double *out_sum,
                       int64_t *out_count) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->factored) return fail(c, BSVD_ESTATE, "sqerr: no factors");
  if (nq < 0 || (nq > 0 && (!u || !i || !y)) || !out_sum || !out_count)
    return fail(c, BSVD_EINVAL, "sqerr: bad arguments");
  const void *du = u, *di = i, *dy = y;
  CK(device_view(c, u, sizeof(int32_t) * nq, c->s_a, &du), "sqerr");
  CK(device_view(c, i, sizeof(int32_t) * nq, c->s_b, &di), "sqerr");
  CK(device_view(c, y, sizeof(float) * nq, c->s_c, &dy), "sqerr");
  CK(c->d_partials.ensure(sizeof(double) * 2 * kSqerrBlocks), "sqerr");
  CK(c->d_rmse.ensure(2 * sizeof(double)), "sqerr");
  PredictArgs a = predict_args(c);
  a.owned_only = 1;
  mark(c, 4);
  CK(launch_sqerr(a, nq, (const int32_t *)du, (const int32_t *)di,
                  (const float *)dy, c->d_partials.as<double>(),
                  c->d_rmse.as<double>(), c->d_err.as<int32_t>(), c->st),
     "sqerr");
  mark(c, 5);
  c->launches += 2;
  double res[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(res, c->d_rmse.p, sizeof res, cudaMemcpyDeviceToHost,
                     c->st), "sqerr");
  bsvd_status s = read_errors(c, "sqerr");
  if (s != BSVD_OK) return s;
  take(c, 4, 4, 5);
  *out_sum = res[0];
  *out_count = (int64_t)res[1];
  return BSVD_OK;
}

bsvd_status bsvd_block_stats(bsvd_ctx *c, int32_t *nblocks, int64_t *counts,
                             float *mu) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->parted) return fail(c, BSVD_ESTATE, "block_stats: no partition");
  if (nblocks) *nblocks = c->nblocks;
  if (counts)
    CK(cudaMemcpyAsync(counts, c->d_counts.p, sizeof(int64_t) * c->nblocks,
                       cudaMemcpyDeviceToHost, c->st), "block_stats");
  if (mu)
    CK(cudaMemcpyAsync(mu, c->d_mu.p, sizeof(float) * c->nblocks,
                       cudaMemcpyDeviceToHost, c->st), "block_stats");
  CK(cudaStreamSynchronize(c->st), "block_stats");
  return BSVD_OK;
}

bsvd_status bsvd_get_block(bsvd_ctx *c, int32_t b, int32_t *mb, int32_t *nb,
                           int32_t *keff, float *mu, double *sigma, float *P,
                           float *V, float *dense) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->parted) return fail(c, BSVD_ESTATE, "get_block: no partition");
  if (b < 0 || b >= c->nblocks) return fail(c, BSVD_EINVAL, "get_block: bad block %d", b);
  const BlockMeta &bm = c->meta[b];
  if ((sigma || P || V) && !c->factored)
    return fail(c, BSVD_ESTATE, "get_block: no factors");
  if (dense && !bm.owned)
    return fail(c, BSVD_EINVAL, "get_block: block %d is not held by this "
                "context (bsvd_set_owned)", b);
  if (mb) *mb = bm.mb;
  if (nb) *nb = bm.nb;
  if (keff) *keff = c->factored ? bm.keff : 0;
  if (mu)
    CK(cudaMemcpyAsync(mu, c->d_mu.as<float>() + b, sizeof(float),
                       cudaMemcpyDeviceToHost, c->st), "get_block");
  std::vector<float> W;
  std::vector<__nv_bfloat16> Wh;
  if (dense && c->w32) {
    W.resize((size_t)bm.s_pad * bm.L_pad);
    CK(cudaMemcpyAsync(W.data(), c->d_W.as<float>() + bm.w_off,
                       sizeof(float) * W.size(), cudaMemcpyDeviceToHost, c->st),
       "get_block");
  } else if (dense) {
    // the BF16 form keeps only the bf16 copy of its blocks
    Wh.resize((size_t)bm.s_pad * bm.L_pad);
    CK(cudaMemcpyAsync(Wh.data(), c->d_VX.as<__nv_bfloat16>() + bm.vx_off,
                       sizeof(__nv_bfloat16) * Wh.size(),
                       cudaMemcpyDeviceToHost, c->st), "get_block");
    W.resize(Wh.size());
    CK(cudaStreamSynchronize(c->st), "get_block");
    for (size_t j = 0; j < Wh.size(); ++j) W[j] = __bfloat162float(Wh[j]);
  }
  std::vector<float> Fs, FL;
  std::vector<double> sg(c->kp);
  if (c->factored && bm.owned && (sigma || P || V)) {
    Fs.resize((size_t)bm.s_pad * c->kp);
    FL.resize((size_t)bm.L_pad * c->kp);
    CK(cudaMemcpyAsync(Fs.data(), c->d_Fs.as<float>() + bm.fs_off,
                       sizeof(float) * Fs.size(), cudaMemcpyDeviceToHost, c->st),
       "get_block");
    CK(cudaMemcpyAsync(FL.data(), c->d_FL.as<float>() + bm.fl_off,
                       sizeof(float) * FL.size(), cudaMemcpyDeviceToHost, c->st),
       "get_block");
    CK(cudaMemcpyAsync(sg.data(), c->d_sigma.as<double>() + (int64_t)b * c->kp,
                       sizeof(double) * c->kp, cudaMemcpyDeviceToHost, c->st),
       "get_block");
  }
  CK(cudaStreamSynchronize(c->st), "get_block");
  const int kp = c->kp, ke = c->factored ? bm.keff : 0;
  if (sigma)
    for (int j = 0; j < ke; ++j) sigma[j] = sg[j];
  // W orientation -> user side P (U_k S_k) and item side V (unit columns)
  if (P || V) {
    for (int j = 0; j < ke; ++j) {
      const double sj = sg[j];
      for (int r = 0; r < bm.mb; ++r) {
        float v = bm.trans ? FL[(size_t)r * kp + j]
                           : (float)(Fs[(size_t)r * kp + j] * sj);
        if (P) P[(size_t)r * ke + j] = v;
      }
      for (int cc = 0; cc < bm.nb; ++cc) {
        float v = bm.trans ? Fs[(size_t)cc * kp + j]
                           : (sj > 0 ? (float)(FL[(size_t)cc * kp + j] / sj) : 0.f);
        if (V) V[(size_t)cc * ke + j] = v;
      }
    }
  }
  if (dense) {
    for (int r = 0; r < bm.mb; ++r)
      for (int cc = 0; cc < bm.nb; ++cc)
        dense[(size_t)r * bm.nb + cc] =
            bm.trans ? W[(size_t)cc * bm.L_pad + r] : W[(size_t)r * bm.L_pad + cc];
  }
  return BSVD_OK;
}

bsvd_status bsvd_reconstruct(bsvd_ctx *c, int32_t b, int32_t add_mean,
                             float *out) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->factored) return fail(c, BSVD_ESTATE, "reconstruct: no factors");
  if (b < 0 || b >= c->nblocks || !out)
    return fail(c, BSVD_EINVAL, "reconstruct: bad arguments");
  const BlockMeta &bm = c->meta[b];
  if (!bm.owned)
    return fail(c, BSVD_EINVAL, "reconstruct: block %d is not held by this "
                "context (bsvd_set_owned)", b);
  const size_t cells = (size_t)bm.mb * bm.nb;
  if (cells == 0) return BSVD_OK;
  float mu = 0.f;
  if (add_mean)
    CK(cudaMemcpyAsync(&mu, c->d_mu.as<float>() + b, sizeof mu,
                       cudaMemcpyDeviceToHost, c->st), "reconstruct");
  CK(cudaStreamSynchronize(c->st), "reconstruct");
  const bool dev_out = is_device_ptr(out);
  float *dst = out;
  if (!dev_out) {
    CK(c->s_out.ensure(sizeof(float) * cells), "reconstruct");
    dst = c->s_out.as<float>();
  }
  CK(launch_reconstruct(c->d_meta.as<BlockMeta>(), bm, b, c->d_Fs.as<float>(),
                        c->d_FL.as<float>(), c->kp, mu, dst,
                        c->d_err.as<int32_t>(), c->st),
     "reconstruct");
  c->launches += 1;
  if (!dev_out)
    CK(cudaMemcpyAsync(out, dst, sizeof(float) * cells, cudaMemcpyDeviceToHost,
                       c->st), "reconstruct");
  return read_errors(c, "reconstruct");
}

bsvd_status bsvd_factor_report(bsvd_ctx *c, int32_t *iters,
                               int32_t *converged, int32_t *sweeps,
                               int64_t *cycles, float *resid,
                               int32_t *products) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->factored) return fail(c, BSVD_ESTATE, "factor_report: no factors");
  std::vector<SolverState> s(c->nblocks);
  CK(cudaMemcpyAsync(s.data(), c->d_state.p, sizeof(SolverState) * c->nblocks,
                     cudaMemcpyDeviceToHost, c->st), "factor_report");
  CK(cudaStreamSynchronize(c->st), "factor_report");
  for (int32_t b = 0; b < c->nblocks; ++b) {
    if (iters) iters[b] = s[b].iters;
    if (converged) converged[b] = s[b].status == kConverged ? 1 : 0;
    if (sweeps) sweeps[b] = s[b].sweeps;
    if (cycles)
      for (int j = 0; j < 3; ++j) cycles[3 * b + j] = s[b].cycles[j];
    if (resid) resid[b] = s[b].resid;
    if (products) products[b] = s[b].products;
  }
  return BSVD_OK;
}

bsvd_status bsvd_phase_times(bsvd_ctx *c, double *ms) {
  if (!c || !ms) return BSVD_EINVAL;
  if (!c->cfg.profile)
    return fail(c, BSVD_ESTATE, "phase_times: profiling is off");
  for (int j = 0; j < 8; ++j) ms[j] = c->phase_ms[j];
  return BSVD_OK;
}

int64_t bsvd_kernel_launches(const bsvd_ctx *c) {
  return c ? c->launches : -1;
}

int32_t bsvd_gram_path(const bsvd_ctx *c) { return c ? c->gram_used : -1; }

int32_t bsvd_loop_form(const bsvd_ctx *c) { return c ? c->last_graph : -1; }

int64_t bsvd_panel_launches(const bsvd_ctx *c) {
  return c ? c->panel_launches : -1;
}

// ---- blocked SGD (Algorithms 1-2) ----------------------------------------

void bsvd_sgd_params_default(bsvd_sgd_params *prm) {
  if (!prm) return;
  prm->a_user = 0.019;
  prm->b_user = 0.019;
  prm->a_item = 0.004;
  prm->b_item = 0.019;
  prm->a_ubias = 0.004;
  prm->b_ubias = 0.019;
  prm->a_ibias = 0.013;
  prm->b_ibias = 0.007;
  prm->delta = 1e-4;
  prm->k = 13;
  prm->max_steps = 100;
  prm->precision = BSVD_SGD_FP64;
}

bsvd_status bsvd_sgd_prepare(bsvd_ctx *c, int64_t nnz, const int32_t *u,
                             const int32_t *i, const float *x) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->parted) return fail(c, BSVD_ESTATE, "sgd_prepare: no partition");
  if (nnz < 0 || nnz >= ((int64_t)1 << 40) || (nnz > 0 && (!u || !i || !x)))
    return fail(c, BSVD_EINVAL, "sgd_prepare: bad arguments");
  for (int32_t j = 0; j < c->q; ++j)
    if (c->cb[j + 1] - c->cb[j] >= ((int64_t)1 << 23))
      return fail(c, BSVD_EINVAL, "sgd_prepare: a block is too wide");
  c->sgd_ready = false;
  c->sgd_trained = false;
  const GridDesc g = c->grid();
  const int32_t nb = c->nblocks;
  const int64_t nbuckets = (int64_t)(c->diag ? c->p : c->q) * c->m;
  const void *du = u, *di = i, *dx = x;
  CK(device_view(c, u, sizeof(int32_t) * nnz, c->s_a, &du), "sgd_prepare");
  CK(device_view(c, i, sizeof(int32_t) * nnz, c->s_b, &di), "sgd_prepare");
  CK(device_view(c, x, sizeof(float) * nnz, c->s_c, &dx), "sgd_prepare");
  const size_t n1 = (size_t)std::max<int64_t>(nnz, 1);
  // bucket counts, then (from the sort on) the list of large buckets
  CK(c->d_sgd_cnt.ensure(sizeof(unsigned long long) * (nbuckets + 1)),
     "sgd_prepare");
  CK(c->d_sgd_off.ensure(sizeof(int64_t) * (nbuckets + 1)), "sgd_prepare");
  CK(c->d_sgd_key.ensure(sizeof(int64_t) * n1), "sgd_prepare");
  CK(c->d_sgd_src.ensure(sizeof(int64_t) * n1), "sgd_prepare");
  CK(c->d_sgd_u.ensure(sizeof(int32_t) * n1), "sgd_prepare");
  CK(c->d_sgd_i.ensure(sizeof(int32_t) * n1), "sgd_prepare");
  CK(c->d_sgd_x.ensure(sizeof(float) * n1), "sgd_prepare");
  CK(c->d_sgd_r.ensure(sizeof(int32_t) * n1), "sgd_prepare");
  CK(c->d_sgd_c.ensure(sizeof(int32_t) * n1), "sgd_prepare");
  CK(c->d_sgd_range.ensure(sizeof(int64_t) * 2 * nb), "sgd_prepare");
  CK(launch_sgd_order(g, nb, nnz, (const int32_t *)du, (const int32_t *)di,
                      (const float *)dx, c->d_sgd_cnt.as<unsigned long long>(),
                      c->d_sgd_off.as<int64_t>(), c->d_sgd_key.as<int64_t>(),
                      c->d_sgd_src.as<int64_t>(), c->d_sgd_u.as<int32_t>(),
                      c->d_sgd_i.as<int32_t>(), c->d_sgd_x.as<float>(),
                      c->d_sgd_r.as<int32_t>(), c->d_sgd_c.as<int32_t>(),
                      c->d_sgd_range.as<int64_t>(), c->d_err.as<int32_t>(),
                      c->st), "sgd_prepare");
  c->launches += nnz > 0 ? 7 : 2;
  bsvd_status s = read_errors(c, "sgd_prepare");
  if (s != BSVD_OK) return s;
  // the diagonal schedule (Figure 2): blocks sharing no block row or column
  std::vector<int32_t> blocks;
  c->sgd_step_off.assign(1, 0);
  if (c->diag) {
    for (int32_t b = 0; b < nb; ++b) blocks.push_back(b);
    c->sgd_step_off.push_back(nb);
  } else if (c->p >= c->q) {
    for (int32_t st = 0; st < c->p; ++st) {
      for (int32_t j = 0; j < c->q; ++j)
        blocks.push_back(((j + st) % c->p) * c->q + j);
      c->sgd_step_off.push_back((int32_t)blocks.size());
    }
  } else {
    for (int32_t st = 0; st < c->q; ++st) {
      for (int32_t r = 0; r < c->p; ++r)
        blocks.push_back(r * c->q + (r + st) % c->q);
      c->sgd_step_off.push_back((int32_t)blocks.size());
    }
  }
  CK(c->d_sgd_blocks.ensure(sizeof(int32_t) * blocks.size()), "sgd_prepare");
  CK(cudaMemcpyAsync(c->d_sgd_blocks.p, blocks.data(),
                     sizeof(int32_t) * blocks.size(), cudaMemcpyHostToDevice,
                     c->st), "sgd_prepare");
  CK(cudaStreamSynchronize(c->st), "sgd_prepare");
  c->sgd_nnz = nnz;
  c->sgd_ready = true;
  return BSVD_OK;
}

static bsvd_status sgd_rmse(bsvd_ctx *c, double *out) {
  double sum = 0.0;
  CK(c->d_partials.ensure(sizeof(double) * kSqerrBlocks), "sgd_train");
  CK(launch_sgd_sqerr(c->sgd_nnz, c->d_sgd_u.as<int32_t>(),
                      c->d_sgd_i.as<int32_t>(), c->d_sgd_x.as<float>(),
                      c->sgd_k, c->d_sgd_P.as<double>(), c->d_sgd_Q.as<double>(),
                      c->d_sgd_bu.as<double>(), c->d_sgd_bi.as<double>(),
                      c->d_partials.as<double>(), c->d_sgd_sum.as<double>(),
                      c->st), "sgd_train");
  c->launches += 2;
  CK(cudaMemcpyAsync(&sum, c->d_sgd_sum.p, sizeof sum, cudaMemcpyDeviceToHost,
                     c->st), "sgd_train");
  CK(cudaStreamSynchronize(c->st), "sgd_train");
  *out = c->sgd_nnz > 0 ? std::sqrt(sum / (double)c->sgd_nnz) : 0.0;
  return BSVD_OK;
}

bsvd_status bsvd_sgd_train(bsvd_ctx *c, const bsvd_sgd_params *prm,
                           const double *P0, const double *Q0, double *rmse,
                           int32_t *steps_run) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->sgd_ready) return fail(c, BSVD_ESTATE, "sgd_train: no sgd_prepare");
  if (!prm || prm->k < 1 || prm->k > 32 || prm->max_steps < 0 ||
      (prm->precision != BSVD_SGD_FP64 && prm->precision != BSVD_SGD_FP32) ||
      !(std::isfinite(prm->a_user) && std::isfinite(prm->b_user) &&
        std::isfinite(prm->a_item) && std::isfinite(prm->b_item) &&
        std::isfinite(prm->a_ubias) && std::isfinite(prm->b_ubias) &&
        std::isfinite(prm->a_ibias) && std::isfinite(prm->b_ibias)) ||
      std::isnan(prm->delta) || !P0 || !Q0)
    return fail(c, BSVD_EINVAL, "sgd_train: bad parameters");
  const int32_t k = prm->k;
  c->sgd_trained = false;
  c->sgd_k = k;
  const size_t pb = sizeof(double) * (size_t)std::max<int64_t>(c->m * k, 1);
  const size_t qb = sizeof(double) * (size_t)std::max<int64_t>(c->n * k, 1);
  CK(c->d_sgd_P.ensure(pb), "sgd_train");
  CK(c->d_sgd_Q.ensure(qb), "sgd_train");
  CK(c->d_sgd_bu.ensure(sizeof(double) * std::max<int64_t>(c->m, 1)), "sgd_train");
  CK(c->d_sgd_bi.ensure(sizeof(double) * std::max<int64_t>(c->n, 1)), "sgd_train");
  CK(c->d_sgd_sum.ensure(sizeof(double)), "sgd_train");
  CK(cudaMemcpyAsync(c->d_sgd_P.p, P0, sizeof(double) * c->m * k,
                     cudaMemcpyDefault, c->st), "sgd_train");
  CK(cudaMemcpyAsync(c->d_sgd_Q.p, Q0, sizeof(double) * c->n * k,
                     cudaMemcpyDefault, c->st), "sgd_train");
  CK(cudaMemsetAsync(c->d_sgd_bu.p, 0, sizeof(double) * c->m, c->st), "sgd_train");
  CK(cudaMemsetAsync(c->d_sgd_bi.p, 0, sizeof(double) * c->n, c->st), "sgd_train");
  const SgdRates r{prm->a_user, prm->b_user, prm->a_item, prm->b_item,
                   prm->a_ubias, prm->b_ubias, prm->a_ibias, prm->b_ibias};
  const bool f32 = prm->precision == BSVD_SGD_FP32;
  const SgdRates32 r32{(float)prm->a_user,  (float)prm->b_user,
                       (float)prm->a_item,  (float)prm->b_item,
                       (float)prm->a_ubias, (float)prm->b_ubias,
                       (float)prm->a_ibias, (float)prm->b_ibias};
  size_t stage = 0;
  if (f32) {
    // float32 rows of k + 1 (factors, bias); the float64 arrays then hold
    // their widened values, which the RMSE, predict and get read
    CK(c->d_sgd_P32.ensure(sizeof(float) * (size_t)std::max<int64_t>(
                               c->m * (k + 1), 1)), "sgd_train");
    CK(c->d_sgd_Q32.ensure(sizeof(float) * (size_t)std::max<int64_t>(
                               c->n * (k + 1), 1)), "sgd_train");
    CK(launch_sgd_narrow(c->m, c->n, k, c->d_sgd_P.as<double>(),
                         c->d_sgd_Q.as<double>(), c->d_sgd_bu.as<double>(),
                         c->d_sgd_bi.as<double>(), c->d_sgd_P32.as<float>(),
                         c->d_sgd_Q32.as<float>(), c->st), "sgd_train");
    CK(launch_sgd_widen(c->m, c->n, k, c->d_sgd_P32.as<float>(),
                        c->d_sgd_Q32.as<float>(), c->d_sgd_P.as<double>(),
                        c->d_sgd_Q.as<double>(), c->d_sgd_bu.as<double>(),
                        c->d_sgd_bi.as<double>(), c->st), "sgd_train");
    c->launches += 2;
    // stage the blocks in shared memory when the largest one fits
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev), "sgd_train");
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                              dev), "sgd_train");
    for (int32_t b = 0; b < c->nblocks; ++b) {
      const int32_t bi = c->diag ? b : b / c->q, bj = c->diag ? b : b % c->q;
      stage = std::max(stage, sgd_stage_bytes(c->rb[bi + 1] - c->rb[bi],
                                              c->cb[bj + 1] - c->cb[bj], k));
    }
    if (stage > (size_t)optin) stage = 0;
  }
  const GridDesc g = c->grid();
  double prev = 0.0;
  bsvd_status s = sgd_rmse(c, &prev);
  if (s != BSVD_OK) return s;
  if (rmse) rmse[0] = prev;
  int32_t ran = 0;
  for (int32_t step = 0; step < prm->max_steps; ++step) {
    for (size_t t = 0; t + 1 < c->sgd_step_off.size(); ++t) {
      const int32_t a = c->sgd_step_off[t], b = c->sgd_step_off[t + 1];
      if (f32)
        CK(launch_sgd_step_f32(g, b - a, c->d_sgd_blocks.as<int32_t>() + a,
                               c->d_sgd_range.as<int64_t>(),
                               c->d_sgd_r.as<int32_t>(),
                               c->d_sgd_c.as<int32_t>(),
                               c->d_sgd_u.as<int32_t>(),
                               c->d_sgd_i.as<int32_t>(),
                               c->d_sgd_x.as<float>(), c->sgd_nnz, k,
                               c->d_sgd_P32.as<float>(),
                               c->d_sgd_Q32.as<float>(), r32, stage,
                               c->d_err.as<int32_t>(), c->st), "sgd_train");
      else
        CK(launch_sgd_step(b - a, c->d_sgd_blocks.as<int32_t>() + a,
                           c->d_sgd_range.as<int64_t>(),
                           c->d_sgd_u.as<int32_t>(), c->d_sgd_i.as<int32_t>(),
                           c->d_sgd_x.as<float>(), c->sgd_nnz, k,
                           c->d_sgd_P.as<double>(), c->d_sgd_Q.as<double>(),
                           c->d_sgd_bu.as<double>(), c->d_sgd_bi.as<double>(),
                           r, c->d_err.as<int32_t>(), c->st), "sgd_train");
      c->launches += 1;
    }
    if (f32) {
      CK(launch_sgd_widen(c->m, c->n, k, c->d_sgd_P32.as<float>(),
                          c->d_sgd_Q32.as<float>(), c->d_sgd_P.as<double>(),
                          c->d_sgd_Q.as<double>(), c->d_sgd_bu.as<double>(),
                          c->d_sgd_bi.as<double>(), c->st), "sgd_train");
      c->launches += 1;
    }
    ++ran;
    double cur = 0.0;
    s = sgd_rmse(c, &cur);
    if (s != BSVD_OK) return s;
    s = read_errors(c, "sgd_train");
    if (s != BSVD_OK) return s;
    if (rmse) rmse[ran] = cur;
    const bool stop = prev - cur < prm->delta;
    prev = cur;
    if (stop) break;
  }
  if (steps_run) *steps_run = ran;
  c->sgd_trained = true;
  return BSVD_OK;
}

bsvd_status bsvd_sgd_predict(bsvd_ctx *c, int64_t nq, const int32_t *u,
                             const int32_t *i, double *yhat) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->sgd_trained) return fail(c, BSVD_ESTATE, "sgd_predict: not trained");
  if (nq < 0 || (nq > 0 && (!u || !i || !yhat)))
    return fail(c, BSVD_EINVAL, "sgd_predict: bad arguments");
  if (nq == 0) return BSVD_OK;
  const void *du, *di;
  CK(device_view(c, u, sizeof(int32_t) * nq, c->s_a, &du), "sgd_predict");
  CK(device_view(c, i, sizeof(int32_t) * nq, c->s_b, &di), "sgd_predict");
  const bool dev_out = is_device_ptr(yhat);
  double *out = yhat;
  if (!dev_out) {
    CK(c->s_out.ensure(sizeof(double) * nq), "sgd_predict");
    out = c->s_out.as<double>();
  }
  CK(launch_sgd_predict(nq, (const int32_t *)du, (const int32_t *)di,
                        c->sgd_k, c->m, c->n, c->d_sgd_P.as<double>(),
                        c->d_sgd_Q.as<double>(), c->d_sgd_bu.as<double>(),
                        c->d_sgd_bi.as<double>(), out, c->d_err.as<int32_t>(),
                        c->st), "sgd_predict");
  c->launches += 1;
  if (!dev_out)
    CK(cudaMemcpyAsync(yhat, out, sizeof(double) * nq, cudaMemcpyDeviceToHost,
                       c->st), "sgd_predict");
  return read_errors(c, "sgd_predict");
}

bsvd_status bsvd_sgd_get(bsvd_ctx *c, double *P, double *Q, double *bu,
                         double *bi) {
  if (!c) return BSVD_EINVAL;
  c->err.clear();
  if (!c->sgd_trained) return fail(c, BSVD_ESTATE, "sgd_get: not trained");
  if (P)
    CK(cudaMemcpyAsync(P, c->d_sgd_P.p, sizeof(double) * c->m * c->sgd_k,
                       cudaMemcpyDefault, c->st), "sgd_get");
  if (Q)
    CK(cudaMemcpyAsync(Q, c->d_sgd_Q.p, sizeof(double) * c->n * c->sgd_k,
                       cudaMemcpyDefault, c->st), "sgd_get");
  if (bu)
    CK(cudaMemcpyAsync(bu, c->d_sgd_bu.p, sizeof(double) * c->m,
                       cudaMemcpyDefault, c->st), "sgd_get");
  if (bi)
    CK(cudaMemcpyAsync(bi, c->d_sgd_bi.p, sizeof(double) * c->n,
                       cudaMemcpyDefault, c->st), "sgd_get");
  CK(cudaStreamSynchronize(c->st), "sgd_get");
  return BSVD_OK;
}

}  // extern "C"
