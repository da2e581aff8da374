// Serving engine of include/cbspmv.h (cbspmv_server_*): resident matrices, a request queue
// with admission by free device memory, and continuous batching of the in-flight
// requests' work on one stream.
//
// The paper motivates its preprocessing cost by repeated products, as in iterative
// solvers (Sec. 4.5); it has no serving system. This engine keeps analysed matrices on
// the device and advances every in-flight request by one step per tick (a solve in its
// inner CG phase by up to inner_steps iterations, which need no host decision):
//   * a y = alpha*A*x + beta*y request needs one product;
//   * a CG request for an SPD matrix solves A x = b by iterative refinement: the true
//     residual r = b - A x and the solution update stay in FP64 (FP64-value product);
//     each correction A d = r is solved by conjugate gradients with the product on
//     reduced-precision values (BF16 storage, FP32 x, y and accumulation) and FP32
//     vectors, until its residual falls by max(inner_tol, 0.3 tol ||b|| / ||r||) (a later
//     correction only needs to close the gap to tol); a solve ends when
//     ||b - A x|| <= tol * ||b|| in FP64. The inner CG is the Chronopoulos-Gear form
//     (1989): the product is w = A r of the current residual, and the step lengths come
//     from r.r and w.r alone (alpha = rr / (wr - beta rr / alpha_prev), beta = rr /
//     rr_prev), with s = A p carried by the recurrence s = w + beta s. An iteration is one
//     product, one dot-product step (w.r) and one fused update (p, s, d, r and the next r.r),
//     one launch fewer than the textbook order (alpha needs p.Ap after the product, beta
//     r.r after the update); in exact arithmetic the iterates are those of textbook CG.
// Per tick, the products of all in-flight requests run as one batched launch of the run
// kernel per value type; the CG vector updates and dot products run as batched kernels
// over all requests; one small device-to-host copy of the requests' scalars decides the
// next step of each request. Results do not depend on the mix: every request's products,
// dot products (fixed per-request block partition, partials added in a fixed order) and
// updates are computed the same way alone or with others.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cbspmv.h"
#include "cb_kernels.h"
#include "cb_noalloc.h"
#include "cb_plan.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

cbspmv_status_t sfail(cbspmv_status_t s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  cb::set_last_error(buf);
  return s;
}

// ---- device side: batched vector steps of CG ----------------------------------------------
constexpr int kMaxSlots = 64;       // requests in flight (one batched launch each step)
constexpr int kMaxMatrices = 1024;  // registered matrices per server
constexpr int kVecBlock = 1024;     // vector elements per block of a batched vector kernel
constexpr int kVecThreads = 256;
// A correction A d = r only has to bring the FP64 residual below tol ||b||: it stops at
// max(inner_tol, kCorSafety * tol ||b|| / ||r||) relative to its start (squared here).
constexpr double kCorSafety2 = 0.3 * 0.3;

// Per-request scalars on the device (one array for all slots, copied back every tick).
struct Scalars {
  double rr, rr_prev, rr0, wr, alpha, beta, rn2, bn2, tol2, tol_in2;
  double tol_cor2;   // squared relative tolerance of the current correction solve
  int done;          // refinement: ||r|| <= tol ||b||
  int inner_done;    // correction solve finished
  int inner_it, inner_cap;
  unsigned arrive;   // blocks of the current vector step that have stored their partial sum
  int pad[3];
};

enum Op : int {
  kOpNone = 0,
  kOpRefinePre,    // x64 += d; r64 = b (before r64 = -A x64 + r64)
  kOpRefineDot,    // partial r64 . r64
  kOpRefineStart,  // r_in = r64; d = p = s = 0; partial r_in . r_in
  kOpWR,           // partial w . r_in (w = A r_in)
  kOpUpdate,       // p = r_in + beta p; s = w + beta s; d += alpha p; r_in -= alpha s;
                   // partial r_in . r_in
};

struct VecDesc {
  int op, slot;
  int64_t n;
  int nblk;              // blocks of this request (ceil(n / kVecBlock))
  double* x64;
  double* r64;
  const double* b64;
  void* d;               // inner vectors: float (mixed precision) or double (FP64 CG)
  void* r;
  void* p;
  void* s;               // A p
  const void* w;         // A r
  double* part;          // nblk partial sums
  int first_outer;       // kOpRefineDot: the first refinement (x = 0, so r = b gives ||b||)
};
struct VecBatch {
  int count;
  int blk_base[kMaxSlots + 1];
  VecDesc v[kMaxSlots];
};

template <class T>
__global__ void __launch_bounds__(kVecThreads) vec_kernel(const __grid_constant__ VecBatch b, Scalars* sc) {
  // A dot-product or update step may be launched as a programmatic dependent of the kernel
  // before it: it waits for that kernel's completion and memory before touching anything,
  // and lets the next step's launch start at once (that step waits in turn).
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  // request of this block: the last q with blk_base[q] <= blockIdx.x
  int lo = 0, hi = b.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.blk_base[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const VecDesc& v = b.v[lo];
  const int blk = (int)blockIdx.x - b.blk_base[lo];
  const int64_t i0 = (int64_t)blk * kVecBlock;
  const int64_t i1 = i0 + kVecBlock < v.n ? i0 + kVecBlock : v.n;
  const Scalars& s = sc[v.slot];
  // the inner steps of a solve whose inner CG has converged do nothing (a tick may run
  // several inner iterations; the device knows when a solve converged, the host later)
  if ((v.op == kOpWR || v.op == kOpUpdate) && s.inner_done) return;
  T* d = static_cast<T*>(v.d);
  T* r = static_cast<T*>(v.r);
  T* p = static_cast<T*>(v.p);
  T* sv = static_cast<T*>(v.s);
  const T* wv = static_cast<const T*>(v.w);
  double acc = 0.0;
  switch (v.op) {
    case kOpRefinePre:
      for (int64_t i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
        v.x64[i] += (double)d[i];
        v.r64[i] = v.b64[i];
      }
      break;
    case kOpRefineDot:
      for (int64_t i = i0 + threadIdx.x; i < i1; i += kVecThreads) acc = fma(v.r64[i], v.r64[i], acc);
      break;
    case kOpRefineStart:
      for (int64_t i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
        const T ri = (T)v.r64[i];
        r[i] = ri;
        p[i] = T(0);
        sv[i] = T(0);
        d[i] = T(0);
        acc = fma((double)ri, (double)ri, acc);
      }
      break;
    // The inner solve's dot products accumulate in the inner vectors' type: FP32 for the
    // mixed-precision solve (an FP64 FMA, or a conversion to FP64, per element would hold
    // GB300's slow FP64 pipe longer than the whole FP32 step; the inner solve only needs a
    // residual reduction of inner_tol), FP64 for the FP64 solve. Each block's sum is FP64.
    case kOpWR: {
      T a = T(0);
      for (int64_t i = i0 + threadIdx.x; i < i1; i += kVecThreads) a = fma(wv[i], r[i], a);
      acc = (double)a;
      break;
    }
    case kOpUpdate: {
      const T al = (T)s.alpha, be = (T)s.beta;
      T a = T(0);
      for (int64_t i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
        const T ri = r[i];
        const T pi = fma(be, p[i], ri);
        const T si = fma(be, sv[i], wv[i]);
        p[i] = pi;
        sv[i] = si;
        d[i] = fma(al, pi, d[i]);
        const T rn = fma(-al, si, ri);
        r[i] = rn;
        a = fma(rn, rn, a);
      }
      acc = (double)a;
      break;
    }
    default:
      break;
  }
  // deterministic block sum: fixed shuffle tree, then the block's warps in order
  __shared__ double ws[kVecThreads / 32];
  __shared__ int last;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (v.op == kOpRefinePre || !v.part) return;   // a step without a sum
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) t += ws[w];
    v.part[blk] = t;
    __threadfence();   // the partial before the arrival count
    last = atomicAdd(&sc[v.slot].arrive, 1u) == (unsigned)v.nblk - 1u;
  }
  __syncthreads();
  // the request's last block to arrive adds the block partials in a fixed order (so the
  // result does not depend on which block is last: thread-strided sums, the shuffle tree,
  // the warps in order) and updates the request's scalars for the step; no block waits
  // for another
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < v.nblk; i += kVecThreads) t += __ldcg(v.part + i);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  __syncthreads();   // (every thread is done with ws)
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x != 0) return;
  t = 0.0;
  for (int w = 0; w < kVecThreads / 32; ++w) t += ws[w];
  Scalars& w = sc[v.slot];
  w.arrive = 0u;
  switch (v.op) {
    case kOpRefineDot:
      w.rn2 = t;
      if (v.first_outer) w.bn2 = t;        // x starts at 0, so the first residual is b
      w.done = (t <= w.tol2 * w.bn2) ? 1 : 0;
      break;
    case kOpRefineStart:
      w.rr = w.rr0 = t;
      w.inner_it = 0;
      w.inner_done = t == 0.0 ? 1 : 0;
      w.tol_cor2 = w.rn2 > 0.0 ? fmax(w.tol_in2, kCorSafety2 * w.tol2 * w.bn2 / w.rn2) : w.tol_in2;
      break;
    case kOpWR: {   // the step lengths from rr = r.r and wr = (A r).r alone
      w.wr = t;
      if (w.inner_it == 0) {
        w.beta = 0.0;
        w.alpha = t != 0.0 ? w.rr / t : 0.0;
      } else {
        w.beta = w.rr_prev != 0.0 ? w.rr / w.rr_prev : 0.0;
        const double den = w.alpha != 0.0 ? t - w.beta * w.rr / w.alpha : 0.0;
        w.alpha = den != 0.0 ? w.rr / den : 0.0;
      }
      break;
    }
    case kOpUpdate:
      w.rr_prev = w.rr;
      w.rr = t;
      w.inner_it += 1;
      w.inner_done = (t <= w.tol_cor2 * w.rr0 || w.inner_it >= w.inner_cap || !(t == t)) ? 1 : 0;
      break;
    default:
      break;
  }
}

// ---- host side -------------------------------------------------------------------------------
// First-fit allocator over one device allocation (the memory budget); 256-byte granules.
class Arena {
 public:
  void reset(size_t cap) {
    cap_ = cap;
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, base = it->first + bytes;
        free_.erase(it);
        if (rest) free_[base] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
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
  size_t used() const { return used_; }
  size_t capacity() const { return cap_; }

 private:
  size_t cap_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

enum Phase { kPhSpmv = 0, kPhRefine, kPhInner };

struct Req {
  uint64_t id = 0;
  cbspmv_request_t q{};
  cbspmv_result_t res{};
  int slot = -1;
  Phase ph = kPhSpmv;
  bool fresh = true;   // admitted this tick: inputs to copy in
  int outer = 0;
  int inner_seen = 0;   // inner iterations of the current correction already counted
  size_t off = 0, bytes = 0;
  // device workspace (inside the arena)
  double *x64 = nullptr, *r64 = nullptr, *b64 = nullptr, *y64 = nullptr;
  void *d = nullptr, *r = nullptr, *p = nullptr, *sv = nullptr, *wv = nullptr;   // inner CG vectors
  void* part_hi = nullptr;   // partial sums of split block rows, FP64-value product
  void* part_lo = nullptr;   // same, inner product
  double* dots = nullptr;
  int nblk = 0;
};

struct Matrix {
  cbspmv_handle_t hi = nullptr;   // FP64 values
  cbspmv_handle_t lo = nullptr;   // inner-solve values (BF16, or FP64 for a plain FP64 CG)
  int64_t m = 0, n = 0;
};

}  // namespace

namespace cb {
// Launch arguments of a product on handle h (capi.cu); partial overrides the handle's
// partial-sum buffer.
bool server_run_args(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta, void* partial,
                     RunArgs* out, int* grid, int* n_slots, int* value_dtype);
}  // namespace cb

struct cbspmv_server_s {
  uint32_t magic = 0xCB5E4E01u;
  cbspmv_server_opts_t o{};
  cudaStream_t stream = nullptr;
  uint8_t* arena_base = nullptr;
  Scalars* d_sc = nullptr;
  Scalars* h_sc = nullptr;          // pinned copy
  Arena arena;
  std::vector<Matrix> mats;   // capacity reserved at creation: the engine reads it unlocked
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;                       // submitted, not admitted
  std::vector<std::shared_ptr<Req>> inflight;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> all;       // by ticket, until taken
  std::atomic<uint64_t> next_id{1};
  bool stop = false;
  std::string engine_error;
  std::thread th;
  int slots_used[kMaxSlots] = {0};
  cbspmv_server_stats_t stats{};

  bool valid() const { return magic == 0xCB5E4E01u; }
  void engine();
  cbspmv_status_t tick(std::vector<std::shared_ptr<Req>>& act, std::string* err);
  bool admit_one(const std::shared_ptr<Req>& r);
  void release(const std::shared_ptr<Req>& r);
};

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static int handle_slots(cbspmv_handle_t h) {
  cb::RunArgs a;
  int g = 0, ns = 0, dt = 0;
  cb::server_run_args(h, nullptr, nullptr, 1.0, 0.0, nullptr, &a, &g, &ns, &dt);
  return ns;
}

// Device workspace of one request of `kind` on matrix M (the layout admit_one carves out of
// the arena): x and y for a product; x, r, b in FP64, the inner CG vectors and the block
// partials for a solve; plus the partial sums of split block rows of each product.
static size_t workspace_bytes(const Matrix& M, int kind, size_t es_in, int* nblk, size_t* part_hi_out,
                              size_t* part_lo_out) {
  const int64_t m = M.m, n = M.n;
  const size_t part_hi = (size_t)std::max(handle_slots(M.hi), 1) * 16 * 8;
  size_t part_lo = 0;
  size_t need = 0;
  *nblk = 0;
  if (kind == CBSPMV_REQ_SPMV) {
    need = align256(n * 8) + align256(m * 8) + align256(part_hi);
  } else {
    part_lo = (size_t)std::max(handle_slots(M.lo), 1) * 16 * es_in;
    *nblk = (int)((n + kVecBlock - 1) / kVecBlock);
    need = 3 * align256(n * 8) + 5 * align256(n * es_in) + align256(part_hi) + align256(part_lo) +
           align256((size_t)std::max(*nblk, 1) * 8);
  }
  if (part_hi_out) *part_hi_out = part_hi;
  if (part_lo_out) *part_lo_out = part_lo;
  return need;
}

bool cbspmv_server_s::admit_one(const std::shared_ptr<Req>& r) {
  const Matrix& M = mats[r->q.matrix];
  const size_t es_in = (o.cg_inner_dtype == CBSPMV_F64) ? 8 : 4;
  const int64_t m = M.m, n = M.n;
  size_t part_hi = 0, part_lo = 0;
  const size_t need = workspace_bytes(M, r->q.kind, es_in, &r->nblk, &part_hi, &part_lo);
  int slot = -1;
  for (int s = 0; s < o.max_inflight && s < kMaxSlots; ++s)
    if (!slots_used[s]) { slot = s; break; }
  if (slot < 0) return false;
  size_t off = 0;
  if (!arena.alloc(need, &off)) return false;
  slots_used[slot] = 1;
  r->slot = slot;
  r->off = off;
  r->bytes = need;
  uint8_t* p = arena_base + off;
  auto take = [&](size_t bytes) { uint8_t* q = p; p += align256(bytes); return q; };
  if (r->q.kind == CBSPMV_REQ_SPMV) {
    r->x64 = (double*)take(n * 8);
    r->y64 = (double*)take(m * 8);
    r->part_hi = take(part_hi);
    r->ph = kPhSpmv;
  } else {
    r->x64 = (double*)take(n * 8);
    r->r64 = (double*)take(n * 8);
    r->b64 = (double*)take(n * 8);
    r->d = take(n * es_in);
    r->r = take(n * es_in);
    r->p = take(n * es_in);
    r->sv = take(n * es_in);
    r->wv = take(n * es_in);
    r->part_hi = take(part_hi);
    r->part_lo = take(part_lo);
    r->dots = (double*)take((size_t)std::max(r->nblk, 1) * 8);
    r->ph = kPhRefine;
  }
  r->fresh = true;
  r->res.t_admit = now_s();
  stats.admitted++;
  return true;
}

void cbspmv_server_s::release(const std::shared_ptr<Req>& r) {
  if (r->slot >= 0) slots_used[r->slot] = 0;
  arena.release(r->off, r->bytes);
  r->slot = -1;
}

// after_kernel: the step directly follows a kernel on the stream (a product or another
// step), so its launch may overlap that kernel's tail (programmatic dependent launch)
template <class T>
static cudaError_t launch_vec(const VecBatch& b, Scalars* sc, cudaStream_t s, bool after_kernel) {
  if (b.count == 0 || b.blk_base[b.count] == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)b.blk_base[b.count]);
  cfg.blockDim = dim3(kVecThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl;
  cfg.numAttrs = after_kernel ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, vec_kernel<T>, b, sc);
}

cbspmv_status_t cbspmv_server_s::tick(std::vector<std::shared_ptr<Req>>& act, std::string* err) {
  cudaStream_t s = stream;
  const bool inner64 = o.cg_inner_dtype == CBSPMV_F64;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && err->empty()) *err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  // 1. inputs of newly admitted requests
  for (auto& r : act) {
    if (!r->fresh) continue;
    const Matrix& M = mats[r->q.matrix];
    Scalars init{};
    if (r->q.kind == CBSPMV_REQ_SPMV) {
      cu(cudaMemcpyAsync(r->x64, r->q.in, M.n * 8, cudaMemcpyHostToDevice, s), "copy x");
      if (r->q.beta != 0.0) cu(cudaMemcpyAsync(r->y64, r->q.out, M.m * 8, cudaMemcpyHostToDevice, s), "copy y");
    } else {
      cu(cudaMemcpyAsync(r->b64, r->q.in, M.n * 8, cudaMemcpyHostToDevice, s), "copy b");
      cu(cudaMemsetAsync(r->x64, 0, M.n * 8, s), "zero x");
      cu(cudaMemsetAsync(r->d, 0, M.n * (inner64 ? 8 : 4), s), "zero d");
      init.tol2 = r->q.tol * r->q.tol;
      init.tol_in2 = o.inner_tol * o.inner_tol;
      init.inner_cap = o.inner_max_iter;
      h_sc[r->slot] = init;
      cu(cudaMemcpyAsync(d_sc + r->slot, &h_sc[r->slot], sizeof(Scalars), cudaMemcpyHostToDevice, s), "copy scalars");
    }
  }
  // 2. refinement pre-step: x += d, r = b
  VecBatch vb{};
  auto add = [&](VecBatch& b, const std::shared_ptr<Req>& r, int op) {
    VecDesc& v = b.v[b.count];
    v = VecDesc{};
    v.op = op;
    v.slot = r->slot;
    v.n = mats[r->q.matrix].n;
    v.nblk = r->nblk;
    v.x64 = r->x64; v.r64 = r->r64; v.b64 = r->b64;
    v.d = r->d; v.r = r->r; v.p = r->p; v.s = r->sv; v.w = r->wv;
    v.part = r->dots;
    b.blk_base[b.count + 1] = b.blk_base[b.count] + r->nblk;
    b.count++;
  };
  auto vec = [&](const VecBatch& b, bool after_kernel) {
    return inner64 ? launch_vec<double>(b, d_sc, s, after_kernel) : launch_vec<float>(b, d_sc, s, after_kernel);
  };
  for (auto& r : act)
    if (r->ph == kPhRefine) add(vb, r, kOpRefinePre);
  cu(vec(vb, false), "refine pre-step");   // (after the input copies)
  // 3. products: FP64 values (y = Ax requests, true residuals), inner values (CG steps)
  std::vector<cb::RunArgs> hi, lo;
  int grid = 0;
  for (auto& r : act) {
    const Matrix& M = mats[r->q.matrix];
    cb::RunArgs a{};
    int g = 0, ns = 0, dt = 0;
    if (r->ph == kPhSpmv) {
      cb::server_run_args(M.hi, r->x64, r->y64, r->q.alpha, r->q.beta, r->part_hi, &a, &g, &ns, &dt);
      if (M.m) hi.push_back(a);
    } else if (r->ph == kPhRefine) {
      cb::server_run_args(M.hi, r->x64, r->r64, -1.0, 1.0, r->part_hi, &a, &g, &ns, &dt);
      if (M.m) hi.push_back(a);
    } else {
      cb::server_run_args(M.lo, r->r, r->wv, 1.0, 0.0, r->part_lo, &a, &g, &ns, &dt);
      if (M.m) lo.push_back(a);
    }
    grid = g;
  }
  if (!hi.empty()) cu(cb::launch_spmv_batch(hi.data(), (int)hi.size(), grid, s), "batched product (FP64)");
  if (!lo.empty()) cu(cb::launch_spmv_batch(lo.data(), (int)lo.size(), grid, s), "batched product (inner)");
  stats.launches += (hi.empty() ? 0 : 1) + (lo.empty() ? 0 : 1);
  // 4. dot products and updates
  // (each vector step's last block per request finishes the step's dot product and the
  // request's scalars: no separate launch)
  VecBatch v1{};
  for (auto& r : act) {
    if (r->ph == kPhRefine) {
      add(v1, r, kOpRefineDot);
      v1.v[v1.count - 1].first_outer = r->outer == 0;
    } else if (r->ph == kPhInner) {
      add(v1, r, kOpWR);
    }
  }
  cu(vec(v1, !hi.empty() || !lo.empty()), "dot step 1");
  // the refinement's convergence is known on the device; requests that continue start or
  // continue their inner solve
  VecBatch v2{};
  for (auto& r : act) {
    if (r->ph == kPhRefine) add(v2, r, kOpRefineStart);   // harmless for a converged request
    else if (r->ph == kPhInner) add(v2, r, kOpUpdate);
  }
  cu(vec(v2, true), "dot step 2");
  // 4b. further inner iterations of the solves in their inner phase: w = A r, the step
  //     lengths from w . r, the updates with r . r; a solve whose inner CG converged
  //     meanwhile skips them (device).
  //     Each solve runs `quota` iterations this tick: all inner_steps, or with
  //     cg_oldest_first inner_steps for the oldest, half for the next, a quarter for the rest
  {
    std::vector<std::pair<int, std::shared_ptr<Req>>> inner;   // (quota, request), oldest first
    for (auto& r : act)
      if (r->ph == kPhInner) {
        const int rank = (int)inner.size();
        const int q = !o.cg_oldest_first || rank == 0 ? o.inner_steps
                      : std::max(1, rank == 1 ? o.inner_steps / 2 : o.inner_steps / 4);
        inner.push_back({q, r});
      }
    std::vector<cb::RunArgs> lo2;
    VecBatch vwr{}, vup{};
    int members = -1;
    for (int it = 1; it < o.inner_steps; ++it) {
      int n = 0;
      for (auto& e : inner) n += e.first > it;
      if (n == 0) break;
      if (n != members) {   // the batches of the solves with iterations left
        members = n;
        lo2.clear();
        vwr = VecBatch{};
        vup = VecBatch{};
        for (auto& e : inner) {
          if (e.first <= it) continue;
          const auto& r = e.second;
          const Matrix& M = mats[r->q.matrix];
          cb::RunArgs a{};
          int g = 0, ns = 0, dt = 0;
          cb::server_run_args(M.lo, r->r, r->wv, 1.0, 0.0, r->part_lo, &a, &g, &ns, &dt);
          if (M.m) lo2.push_back(a);
          grid = g;
          add(vwr, r, kOpWR);
          add(vup, r, kOpUpdate);
        }
      }
      if (!lo2.empty()) cu(cb::launch_spmv_batch(lo2.data(), (int)lo2.size(), grid, s), "batched product (inner)");
      stats.launches += lo2.empty() ? 0 : 1;
      cu(vec(vwr, !lo2.empty()), "inner w.r");
      cu(vec(vup, true), "inner update");
    }
  }
  // 5. scalars back to the host, then decide every request's next step
  cu(cudaMemcpyAsync(h_sc, d_sc, sizeof(Scalars) * kMaxSlots, cudaMemcpyDeviceToHost, s), "copy scalars back");
  cu(cudaStreamSynchronize(s), "tick");
  if (!err->empty()) return CBSPMV_ERR_CUDA;
  std::vector<std::shared_ptr<Req>> finished;
  for (auto& r : act) {
    r->fresh = false;
    const Scalars& sc = h_sc[r->slot];
    if (r->ph == kPhSpmv) {
      finished.push_back(r);
    } else if (r->ph == kPhRefine) {
      r->res.rel_residual = sc.bn2 > 0 ? std::sqrt(sc.rn2 / sc.bn2) : 0.0;
      if (sc.done || sc.bn2 == 0.0) {
        r->res.status = CBSPMV_OK;
        finished.push_back(r);
      } else if (r->outer >= o.max_outer) {
        r->res.status = CBSPMV_ERR_TIMEOUT;     // did not reach the tolerance in max_outer refinements
        finished.push_back(r);
      } else {
        r->outer++;
        r->res.refinements = r->outer;
        r->ph = sc.inner_done ? kPhRefine : kPhInner;
        r->inner_seen = 0;    // the refinement start reset the device's count
      }
    } else {
      r->res.iterations += sc.inner_it - r->inner_seen;
      r->inner_seen = sc.inner_it;
      if (sc.inner_done) r->ph = kPhRefine;
    }
  }
  // results of finished requests to the host
  for (auto& r : finished) {
    const Matrix& M = mats[r->q.matrix];
    if (r->q.kind == CBSPMV_REQ_SPMV) {
      cu(cudaMemcpyAsync(r->q.out, r->y64, M.m * 8, cudaMemcpyDeviceToHost, s), "copy y back");
      r->res.status = CBSPMV_OK;
    } else {
      cu(cudaMemcpyAsync(r->q.out, r->x64, M.n * 8, cudaMemcpyDeviceToHost, s), "copy x back");
    }
  }
  if (!finished.empty()) cu(cudaStreamSynchronize(s), "result copies");
  if (!err->empty()) return CBSPMV_ERR_CUDA;
  const double t = now_s();
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& r : finished) {
      r->res.t_done = t;
      r->res.done = 1;
      release(r);
      stats.completed++;
      inflight.erase(std::find(inflight.begin(), inflight.end(), r));
    }
    stats.ticks++;
  }
  if (!finished.empty()) cv_done.notify_all();
  return CBSPMV_OK;
}

void cbspmv_server_s::engine() {
  cudaSetDevice(o.device);
  for (;;) {
    std::vector<std::shared_ptr<Req>> act;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop || !queue.empty() || !inflight.empty(); });
      if (stop) break;
      // admission in arrival order while a slot and memory are free; a CG request beyond
      // the limit on solves in flight keeps its place, later products go past it
      int cg_in = 0;
      for (auto& r : inflight) cg_in += r->q.kind == CBSPMV_REQ_CG;
      const int cg_cap = o.max_inflight_cg > 0 ? o.max_inflight_cg : kMaxSlots;
      for (auto it = queue.begin(); it != queue.end();) {
        const bool cg = (*it)->q.kind == CBSPMV_REQ_CG;
        if (cg && cg_in >= cg_cap) {
          ++it;
          continue;
        }
        if (!admit_one(*it)) break;
        cg_in += cg;
        inflight.push_back(*it);
        it = queue.erase(it);
      }
      act = inflight;
      stats.max_inflight_seen = std::max<int64_t>(stats.max_inflight_seen, (int64_t)act.size());
      stats.arena_used_max = std::max<int64_t>(stats.arena_used_max, (int64_t)arena.used());
    }
    if (act.empty()) continue;
    std::string err;
    if (tick(act, &err) != CBSPMV_OK) {
      std::lock_guard<std::mutex> lk(mu);
      engine_error = err;
      for (auto& r : inflight) {
        r->res.done = 1;
        r->res.status = CBSPMV_ERR_CUDA;
        r->res.t_done = now_s();
      }
      inflight.clear();
      for (auto& r : queue) {
        r->res.done = 1;
        r->res.status = CBSPMV_ERR_CUDA;
        r->res.t_done = now_s();
      }
      queue.clear();
      cv_done.notify_all();
      break;
    }
  }
}

namespace cb {
bool server_valid(cbspmv_server_t s) { return s && s->valid(); }
}

extern "C" {

cbspmv_status_t cbspmv_server_default_opts(cbspmv_server_opts_t* o) {
  if (!o) return sfail(CBSPMV_ERR_INVALID, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->memory_budget = (int64_t)4 << 30;
  o->max_inflight = kMaxSlots;
  o->cg_inner_dtype = CBSPMV_BF16;
  o->inner_tol = 1e-4;
  o->inner_max_iter = 2000;
  o->max_outer = 30;
  o->inner_steps = 8;
  cb::set_last_error("");
  return CBSPMV_OK;
}

cbspmv_status_t cbspmv_server_create(const cbspmv_server_opts_t* opts, cbspmv_server_t* out) {
  if (!out) return sfail(CBSPMV_ERR_INVALID, "out is NULL");
  *out = nullptr;
  cbspmv_server_opts_t o;
  if (opts) o = *opts; else cbspmv_server_default_opts(&o);
  if (o.max_inflight < 1 || o.max_inflight > kMaxSlots)
    return sfail(CBSPMV_ERR_INVALID, "max_inflight must be in [1, %d]", kMaxSlots);
  if (o.memory_budget < (1 << 20)) return sfail(CBSPMV_ERR_INVALID, "memory_budget below 1 MiB");
  if (o.cg_inner_dtype < CBSPMV_F64 || o.cg_inner_dtype > CBSPMV_F16)
    return sfail(CBSPMV_ERR_INVALID, "unknown cg_inner_dtype");
  if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0) || o.inner_max_iter < 1 || o.max_outer < 1)
    return sfail(CBSPMV_ERR_INVALID, "inner_tol in (0, 1), inner_max_iter >= 1, max_outer >= 1");
  if (o.inner_steps < 0 || o.inner_steps > 64) return sfail(CBSPMV_ERR_INVALID, "inner_steps must be in [0, 64]");
  if (o.max_inflight_cg < 0 || o.max_inflight_cg > kMaxSlots)
    return sfail(CBSPMV_ERR_INVALID, "max_inflight_cg must be in [0, %d]", kMaxSlots);
  if (o.cg_oldest_first != 0 && o.cg_oldest_first != 1) return sfail(CBSPMV_ERR_INVALID, "cg_oldest_first must be 0 or 1");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return sfail(CBSPMV_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  if (o.device < 0 || o.device >= ndev) return sfail(CBSPMV_ERR_INVALID, "device %d not present", o.device);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(o.device);
  auto* s = new (std::nothrow) cbspmv_server_s();
  if (!s) return sfail(CBSPMV_ERR_OOM, "host allocation failed");
  if (o.inner_steps == 0) o.inner_steps = 8;
  s->o = o;
  e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->arena_base, (size_t)o.memory_budget);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_sc, sizeof(Scalars) * kMaxSlots);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_sc, sizeof(Scalars) * kMaxSlots);
  if (e == cudaSuccess) e = cudaMemset(s->d_sc, 0, sizeof(Scalars) * kMaxSlots);
  if (e != cudaSuccess) {
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->d_sc) cudaFree(s->d_sc);
    if (s->h_sc) cudaFreeHost(s->h_sc);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    cudaSetDevice(prev);
    return sfail(e == cudaErrorMemoryAllocation ? CBSPMV_ERR_OOM : CBSPMV_ERR_CUDA, "server set-up: %s",
                 cudaGetErrorString(e));
  }
  s->arena.reset((size_t)o.memory_budget);
  s->mats.reserve(kMaxMatrices);
  s->th = std::thread([s] { s->engine(); });
  cudaSetDevice(prev);
  *out = s;
  cb::set_last_error("");
  return CBSPMV_OK;
}

cbspmv_status_t cbspmv_server_register(cbspmv_server_t s, const cbspmv_csr_t* A, const cbspmv_opts_t* opts,
                                       int* matrix_id) {
  if (!cb::server_valid(s) || !A || !matrix_id) return sfail(CBSPMV_ERR_INVALID, "invalid server or NULL argument");
  cbspmv_opts_t o;
  if (opts) o = *opts; else cbspmv_default_opts(&o);
  o.device = s->o.device;
  Matrix M;
  M.m = A->m;
  M.n = A->n;
  o.value_dtype = CBSPMV_F64;
  cbspmv_status_t st = cbspmv_analyze(A, &o, s->stream, &M.hi);
  if (st != CBSPMV_OK) return st;
  if (A->m == A->n) {    // square: CG requests possible; analyse the inner-solve values too
    o.value_dtype = s->o.cg_inner_dtype;
    if (o.record_layout == 0) o.record_layout = 2;   // lane streams for the inner values too
    st = cbspmv_analyze(A, &o, s->stream, &M.lo);
    if (st != CBSPMV_OK) {
      cbspmv_destroy(M.hi);
      return st;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->mats.size() >= kMaxMatrices) {
    cbspmv_destroy(M.hi);
    cbspmv_destroy(M.lo);
    return sfail(CBSPMV_ERR_INVALID, "at most %d matrices per server", kMaxMatrices);
  }
  s->mats.push_back(M);
  *matrix_id = (int)s->mats.size() - 1;
  cb::set_last_error("");
  return CBSPMV_OK;
}

cbspmv_status_t cbspmv_server_submit(cbspmv_server_t s, const cbspmv_request_t* q, uint64_t* ticket) {
  if (!cb::server_valid(s) || !q || !ticket) return sfail(CBSPMV_ERR_INVALID, "invalid server or NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (q->matrix < 0 || q->matrix >= (int)s->mats.size()) return sfail(CBSPMV_ERR_INVALID, "unknown matrix %d", q->matrix);
  const Matrix& M = s->mats[q->matrix];
  if ((!q->in && M.n) || (!q->out && (q->kind == CBSPMV_REQ_CG ? M.n : M.m)))
    return sfail(CBSPMV_ERR_INVALID, "NULL input or output");
  if (q->kind == CBSPMV_REQ_CG) {
    if (!M.lo) return sfail(CBSPMV_ERR_INVALID, "CG needs a square matrix");
    if (!(q->tol > 0.0)) return sfail(CBSPMV_ERR_INVALID, "CG tolerance must be > 0");
  } else if (q->kind != CBSPMV_REQ_SPMV) {
    return sfail(CBSPMV_ERR_INVALID, "unknown request kind");
  }
  if (!s->engine_error.empty()) return sfail(CBSPMV_ERR_CUDA, "server stopped: %s", s->engine_error.c_str());
  {
    // a request that would not fit the whole memory budget could never be admitted and
    // would hold every later request behind it in the arrival-order queue
    const size_t es_in = (s->o.cg_inner_dtype == CBSPMV_F64) ? 8 : 4;
    int nblk = 0;
    const size_t need = workspace_bytes(M, q->kind, es_in, &nblk, nullptr, nullptr);
    if (need > s->arena.capacity())
      return sfail(CBSPMV_ERR_OOM, "request needs %zu bytes of workspace, the memory budget holds %zu", need,
                   s->arena.capacity());
  }
  auto r = std::make_shared<Req>();
  r->id = s->next_id++;
  r->q = *q;
  r->res.t_submit = now_s();
  r->res.status = CBSPMV_OK;
  s->queue.push_back(r);
  s->all[r->id] = r;
  s->stats.submitted++;
  *ticket = r->id;
  s->cv_work.notify_one();
  cb::set_last_error("");
  return CBSPMV_OK;
}

static cbspmv_status_t take_result(cbspmv_server_t s, uint64_t ticket, cbspmv_result_t* res, bool* found) {
  auto it = s->all.find(ticket);
  *found = it != s->all.end();
  if (!*found) return sfail(CBSPMV_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  *res = it->second->res;
  if (res->done) s->all.erase(it);
  return CBSPMV_OK;
}

cbspmv_status_t cbspmv_server_poll(cbspmv_server_t s, uint64_t ticket, cbspmv_result_t* res) {
  if (!cb::server_valid(s) || !res) return sfail(CBSPMV_ERR_INVALID, "invalid server or NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  bool found;
  return take_result(s, ticket, res, &found);
}

cbspmv_status_t cbspmv_server_wait(cbspmv_server_t s, uint64_t ticket, int timeout_ms, cbspmv_result_t* res) {
  if (!cb::server_valid(s) || !res) return sfail(CBSPMV_ERR_INVALID, "invalid server or NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return sfail(CBSPMV_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                      [&] { return r->res.done != 0; });
  *res = r->res;
  if (!ok) return sfail(CBSPMV_ERR_TIMEOUT, "request %llu not done within %d ms", (unsigned long long)ticket, timeout_ms);
  s->all.erase(ticket);
  cb::set_last_error("");
  return CBSPMV_OK;
}

cbspmv_status_t cbspmv_server_get_stats(cbspmv_server_t s, cbspmv_server_stats_t* st) {
  if (!cb::server_valid(s) || !st) return sfail(CBSPMV_ERR_INVALID, "invalid server or NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->stats;
  st->arena_capacity = (int64_t)s->arena.capacity();
  st->queued = (int64_t)s->queue.size();
  st->inflight = (int64_t)s->inflight.size();
  return CBSPMV_OK;
}

cbspmv_status_t cbspmv_server_destroy(cbspmv_server_t s) {
  if (!s) return CBSPMV_OK;
  if (!cb::server_valid(s)) return sfail(CBSPMV_ERR_INVALID, "invalid server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->o.device);
  cudaStreamSynchronize(s->stream);
  for (auto& M : s->mats) {
    cbspmv_destroy(M.hi);
    cbspmv_destroy(M.lo);
  }
  cudaFree(s->arena_base);
  cudaFree(s->d_sc);
  cudaFreeHost(s->h_sc);
  cudaStreamDestroy(s->stream);
  cudaSetDevice(prev);
  s->magic = 0;
  delete s;
  return CBSPMV_OK;
}

}  // extern "C"
