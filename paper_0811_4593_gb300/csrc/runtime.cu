// runtime.cu -- the C ABI declared in include/lbm.h: context lifetime, validation of
// the boundary specification, device buffers (through the allocator hook), stream
// handling and dispatch to the kernels of the context's storage precision.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "d3q19.cuh"
#include "lbm_internal.h"

namespace {

lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_release = nullptr;
void* g_user = nullptr;
thread_local std::string g_err = "no error";

struct Allocation {
  void* ptr;     // start of the allocation (the leading guard)
  size_t bytes;  // bytes handed out, between the two guards
};

// Every context buffer sits between two guard regions filled with GUARD_BYTE when it is
// allocated; lbm_check_guards reads them back, so a write just outside a buffer (the
// kind an index error makes) is caught without a device-side sanitizer.
constexpr size_t GUARD = 256;
constexpr unsigned char GUARD_BYTE = 0xa5;

}  // namespace

struct lbm_ctx {
  int device = 0;
  int nx = 0, ny = 0, nz = 0;
  uint32_t N = 0;
  double tau = 1.0, rho0 = 1.0;
  lbm_precision prec = LBM_F32;
  lbm_scheme scheme = LBM_SCHEME_AB;
  lbm::SweepArgs args{};
  void* buf[2] = {nullptr, nullptr};  // AA: both entries are the one population array
  int cur = 0;  // A/B: buf[cur] holds the current post-collision state
  void* snap = nullptr;
  double* partials = nullptr;
  double* dred = nullptr;
  uint32_t* derr = nullptr;  // device error word of the sweeps (SweepArgs::err)
  cudaStream_t stream = nullptr;
  int64_t steps = 0, launches = 0, device_bytes = 0;
  std::string err = "no error";
  lbm_alloc_fn alloc = nullptr;
  lbm_free_fn release = nullptr;
  void* user = nullptr;
  std::vector<Allocation> allocations;
  lbm_batch* batch = nullptr;  // batch the context is attached to, if any
  int batch_slot = -1;
};

struct lbm_batch {
  int device = 0;
  int capacity = 0;
  lbm_precision prec = LBM_F32;
  int scheme = -1;  // scheme of the attached contexts (-1: none attached yet)
  std::vector<lbm_ctx*> slots;
  std::vector<uint8_t> has_result;  // slot took part in the last residual step
  lbm::BatchHeader* h_hdr = nullptr;  // pinned host mirror of the device table
  lbm::BatchEntry* h_ent = nullptr;
  double* h_res = nullptr;            // pinned [capacity][4]
  lbm::BatchHeader* d_hdr = nullptr;
  lbm::BatchEntry* d_ent = nullptr;
  double* d_res = nullptr;
  lbm::BatchChunk* h_chunks = nullptr;  // pinned mirror of the chunk table
  lbm::BatchChunk* d_chunks = nullptr;
  uint32_t* d_next = nullptr;           // chunk counter of the batched sweep
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t table_free = nullptr;  // the last table upload has read the host mirror
  int grid = 0;  // persistent grid of every batched launch
  uint32_t total_blocks = 0;
  struct Graph {
    int n;
    bool resid;
    int scheme;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  bool results_valid = false;
  int64_t steps = 0, launches = 0, device_bytes = 0;
  std::string err = "no error";
  lbm_alloc_fn alloc = nullptr;
  lbm_free_fn release = nullptr;
  void* user = nullptr;
  std::vector<Allocation> allocations;
};

namespace {

size_t storage_bytes(lbm_precision p) { return p == LBM_F64 ? 8 : (p == LBM_F32 ? 4 : 2); }
size_t compute_bytes(lbm_precision p) { return p == LBM_F64 ? 8 : 4; }

lbm_status fail(lbm_ctx* ctx, lbm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  g_err = buf;
  return st;
}

lbm_status cuda_fail(lbm_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s (%s)", what,
              cudaGetErrorString(e), cudaGetErrorName(e));
}

#define LBM_CUDA(ctx, expr, what)                      \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

// Makes the context's device current for the scope of one ABI call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

void* ctx_alloc(lbm_ctx* ctx, size_t bytes) {
  void* p = nullptr;
  const size_t total = bytes + 2 * GUARD;
  if (ctx->alloc) {
    p = ctx->alloc(total, ctx->user);
  } else if (cudaMalloc(&p, total) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) return nullptr;
  if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
    // the sweeps' 16-byte bulk copies and pair loads need aligned buffers
    if (ctx->release) ctx->release(p, ctx->user);
    else cudaFree(p);
    fail(ctx, LBM_ERR_OOM, "the allocator hook returned %p, which is not 256-byte aligned", p);
    return nullptr;
  }
  char* base = static_cast<char*>(p);
  if (cudaMemset(base, GUARD_BYTE, GUARD) != cudaSuccess ||
      cudaMemset(base + GUARD + bytes, GUARD_BYTE, GUARD) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->release) ctx->release(p, ctx->user);
    else cudaFree(p);
    return nullptr;
  }
  ctx->allocations.push_back({p, bytes});
  ctx->device_bytes += int64_t(bytes);
  return base + GUARD;
}

void ctx_free_all(lbm_ctx* ctx) {
  for (auto it = ctx->allocations.rbegin(); it != ctx->allocations.rend(); ++it) {
    if (ctx->release) ctx->release(it->ptr, ctx->user);
    else cudaFree(it->ptr);
  }
  ctx->allocations.clear();
  ctx->device_bytes = 0;
}

// Sweep record of one node of face f. Velocity face: u in double and float and
// 1 / (1 - u.n) in double (n the inward normal; |u.n| < 1 is validated). Pressure
// face: the tangential part of u and, in the `inv` field, the prescribed density.
lbm::FaceNode face_node(int f, const double* u, bool pressure, double rho) {
  lbm::FaceNode n{};
  for (int j = 0; j < 3; ++j) n.u[j] = (pressure && j == f / 2) ? 0.0 : u[j];
  for (int j = 0; j < 3; ++j) n.uf[j] = float(n.u[j]);
  const double un = (f % 2 == 0 ? 1.0 : -1.0) * u[f / 2];
  n.inv = pressure ? rho : 1.0 / (1.0 - un);
  n.pad = 0.0f;
  return n;
}

int face_n1(int face, int nx, int ny) { return (face / 2 == 0) ? ny : nx; }
int face_n2(int face, int ny, int nz) { return (face / 2 == 2) ? ny : nz; }

lbm_status validate(int nx, int ny, int nz, double tau, const lbm_face_spec* faces, int prec, double rho0) {
  if (!faces) return fail(nullptr, LBM_ERR_ARG, "faces is NULL");
  if (nx < 3 || ny < 3 || nz < 3) return fail(nullptr, LBM_ERR_ARG, "every dimension must be >= 3 (got %d x %d x %d)", nx, ny, nz);
  const unsigned long long n = 1ull * nx * ny * nz;
  if (19ull * n >= (1ull << 32)) return fail(nullptr, LBM_ERR_ARG, "lattice too large: 19 * %llu populations >= 2^32", n);
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, LBM_ERR_ARG, "tau must be finite and > 1/2 (got %g)", tau);
  if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail(nullptr, LBM_ERR_ARG, "rho0 must be finite and > 0 (got %g)", rho0);
  if (prec < LBM_F64 || prec > LBM_F16_SHIFTED) return fail(nullptr, LBM_ERR_ARG, "unknown precision %d", prec);
  int pressure_axes = 0;
  for (int a = 0; a < 3; ++a) {
    const int k0 = faces[2 * a].kind, k1 = faces[2 * a + 1].kind;
    for (int k : {k0, k1})
      if (k != LBM_FACE_PERIODIC && k != LBM_FACE_VELOCITY && k != LBM_FACE_PRESSURE)
        return fail(nullptr, LBM_ERR_ARG, "axis %d: unknown face kind %d", a, k);
    if ((k0 == LBM_FACE_PERIODIC) != (k1 == LBM_FACE_PERIODIC))
      return fail(nullptr, LBM_ERR_ARG, "axis %d: periodic faces must come in pairs", a);
    if (k0 == LBM_FACE_PRESSURE || k1 == LBM_FACE_PRESSURE) ++pressure_axes;
  }
  if (pressure_axes > 1)
    return fail(nullptr, LBM_ERR_ARG, "pressure faces may lie on one axis only (an edge borders at most one)");
  auto finite3 = [](const double* u) { return std::isfinite(u[0]) && std::isfinite(u[1]) && std::isfinite(u[2]); };
  for (int f = 0; f < 6; ++f) {
    const int kind = faces[f].kind;
    if (kind == LBM_FACE_PERIODIC) continue;
    const int a = f / 2;
    const double sg = (f % 2 == 0) ? 1.0 : -1.0;
    const size_t m = size_t(face_n1(f, nx, ny)) * face_n2(f, ny, nz);
    if (faces[f].u_table) {
      for (size_t i = 0; i < m; ++i) {
        const double* u = faces[f].u_table + 3 * i;
        if (!finite3(u)) return fail(nullptr, LBM_ERR_ARG, "face %d: non-finite velocity at table entry %zu", f, i);
        if (kind == LBM_FACE_VELOCITY && !(std::fabs(sg * u[a]) < 1.0))
          return fail(nullptr, LBM_ERR_ARG, "face %d: |u.n| >= 1 at table entry %zu", f, i);
      }
    } else {
      if (!finite3(faces[f].u)) return fail(nullptr, LBM_ERR_ARG, "face %d: non-finite velocity", f);
      if (kind == LBM_FACE_VELOCITY && !(std::fabs(faces[f].u[a]) < 1.0))
        return fail(nullptr, LBM_ERR_ARG, "face %d: |u.n| >= 1", f);
    }
    if (kind == LBM_FACE_PRESSURE) {
      if (faces[f].rho_table) {
        for (size_t i = 0; i < m; ++i) {
          const double r = faces[f].rho_table[i];
          if (!(r > 0.0) || !std::isfinite(r))
            return fail(nullptr, LBM_ERR_ARG, "face %d: density must be finite and > 0 at table entry %zu", f, i);
        }
      } else if (!(faces[f].rho > 0.0) || !std::isfinite(faces[f].rho)) {
        return fail(nullptr, LBM_ERR_ARG, "face %d: density must be finite and > 0 (got %g)", f, faces[f].rho);
      }
    }
  }
  return LBM_OK;
}

// Point the sweep at buf[from] -> buf[from ^ 1], with the per-population starts.
void set_direction(lbm_ctx* ctx, int from) {
  const size_t es = storage_bytes(ctx->prec);
  const char* src = static_cast<const char*>(ctx->buf[from]);
  char* dst = static_cast<char*>(ctx->buf[from ^ 1]);
  ctx->args.src = src;
  ctx->args.dst = dst;
  for (int k = 0; k < 19; ++k) {
    ctx->args.src_pop[k] = src + size_t(k) * ctx->N * es;
    ctx->args.dst_pop[k] = dst + size_t(k) * ctx->N * es;
  }
}

// Streaming mode of the context's next step: A/B pull, or for AA the gather-scatter
// step after an even number of steps and the in-place step after an odd one.
int next_mode(const lbm_ctx* ctx) {
  if (ctx->scheme == LBM_SCHEME_AB) return 0;
  return (ctx->steps % 2 == 0) ? 1 : 2;
}

cudaError_t dispatch_sweep(lbm_ctx* ctx, bool resid) {
  const int mode = next_mode(ctx);
  switch (ctx->prec) {
    case LBM_F64: return lbm::launch_sweep<double>(ctx->args, resid, mode, ctx->stream);
    case LBM_F32: return lbm::launch_sweep<float>(ctx->args, resid, mode, ctx->stream);
    default: return lbm::launch_sweep<__half>(ctx->args, resid, mode, ctx->stream);
  }
}

// Observations (macros, residual, population copies) need the post-collision state:
// always for A/B, between step pairs for AA (where population k sits in slot -k).
lbm_status require_observable(lbm_ctx* ctx) {
  if (ctx->scheme == LBM_SCHEME_AA && ctx->steps % 2 != 0)
    return fail(ctx, LBM_ERR_STATE, "an AA lattice is observable only after an even number of steps");
  return LBM_OK;
}

cudaError_t dispatch_init(lbm_ctx* ctx, void* dst) {
  switch (ctx->prec) {
    case LBM_F64: return lbm::launch_init<double>(dst, ctx->N, ctx->rho0, ctx->stream);
    case LBM_F32: return lbm::launch_init<float>(dst, ctx->N, ctx->rho0, ctx->stream);
    default: return lbm::launch_init<__half>(dst, ctx->N, ctx->rho0, ctx->stream);
  }
}

lbm_status ensure_reduction_buffers(lbm_ctx* ctx) {
  if (ctx->snap) return LBM_OK;
  const size_t snap_bytes = 3ull * ctx->N * compute_bytes(ctx->prec);
  void* snap = ctx_alloc(ctx, snap_bytes);
  if (!snap) return fail(ctx, LBM_ERR_OOM, "allocation of %zu bytes for the velocity snapshot failed", snap_bytes);
  const size_t part_bytes = 4ull * lbm::sweep_blocks(ctx->N) * sizeof(double);
  void* part = ctx_alloc(ctx, part_bytes);
  if (!part) return fail(ctx, LBM_ERR_OOM, "allocation of %zu bytes for reduction partials failed", part_bytes);
  LBM_CUDA(ctx, cudaMemsetAsync(snap, 0, snap_bytes, ctx->stream), "clearing the velocity snapshot");
  ctx->snap = snap;
  ctx->partials = static_cast<double*>(part);
  ctx->args.snap = snap;
  ctx->args.partials = ctx->partials;
  return LBM_OK;
}

// Work of an attached context is issued on its batch's stream: wait for it before the
// context is used on its own.
lbm_status settle(lbm_ctx* ctx) {
  if (ctx->batch) LBM_CUDA(ctx, cudaStreamSynchronize(ctx->batch->stream), "waiting for the context's batch");
  return LBM_OK;
}

// Final fold of the partial sums and the host-side residual.
// Reads (and clears) the sweeps' device error word after synchronising the stream: a
// sweep that gave up waiting for its staged loads left results that are not valid.
lbm_status check_device_error(lbm_ctx* ctx) {
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronisation");
  if (!ctx->derr) return LBM_OK;
  uint32_t v = 0;
  LBM_CUDA(ctx, cudaMemcpyAsync(&v, ctx->derr, sizeof v, cudaMemcpyDeviceToHost, ctx->stream), "reading the error word");
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "reading the error word");
  if (v == 0) return LBM_OK;
  LBM_CUDA(ctx, cudaMemsetAsync(ctx->derr, 0, sizeof v, ctx->stream), "clearing the error word");
  return fail(ctx, LBM_ERR_CUDA,
              "a sweep gave up waiting for its staged row copies (device error word 0x%x): the state is not valid", v);
}

lbm_status finish_reduction(lbm_ctx* ctx, double* residual, double* mass) {
  LBM_CUDA(ctx, lbm::launch_final_reduce(ctx->partials, lbm::sweep_blocks(ctx->N), ctx->dred, ctx->stream),
           "final reduction launch");
  ctx->launches += 1;
  double h[4];
  LBM_CUDA(ctx, cudaMemcpyAsync(h, ctx->dred, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "reading reductions");
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "synchronising after reductions");
  if (lbm_status st = check_device_error(ctx); st != LBM_OK) return st;
  const double r = h[2] > 0.0 ? std::sqrt(h[1]) / std::sqrt(h[2]) : std::sqrt(h[1]);
  if (residual) *residual = r;
  if (mass) *mass = h[0];
  if (h[3] != 0.0 || !std::isfinite(h[0]) || !std::isfinite(r))
    return fail(ctx, LBM_ERR_DIVERGED, "diverged: %.0f nodes with non-finite or non-positive density or "
                "non-finite velocity (mass %g)", h[3], h[0]);
  return LBM_OK;
}

}  // namespace

namespace lbm {
void record_error(const char* msg) { g_err = msg; }
}  // namespace lbm

extern "C" {

lbm_status lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void* user) {
  if (alloc && !release) return fail(nullptr, LBM_ERR_ARG, "an allocator needs a matching release function");
  g_alloc = alloc;
  g_release = alloc ? release : nullptr;
  g_user = alloc ? user : nullptr;
  return LBM_OK;
}

lbm_status lbm_create(int nx, int ny, int nz, double tau, const lbm_face_spec faces[6], lbm_precision prec,
                      double rho0, lbm_ctx** out) {
  return lbm_create_scheme(nx, ny, nz, tau, faces, prec, rho0, LBM_SCHEME_AB, out);
}

lbm_status lbm_create_scheme(int nx, int ny, int nz, double tau, const lbm_face_spec faces[6], lbm_precision prec,
                             double rho0, lbm_scheme scheme, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (scheme != LBM_SCHEME_AB && scheme != LBM_SCHEME_AA) return fail(nullptr, LBM_ERR_ARG, "unknown scheme %d", int(scheme));
  lbm_status st = validate(nx, ny, nz, tau, faces, prec, rho0);
  if (st != LBM_OK) return st;
  lbm_ctx* ctx = new (std::nothrow) lbm_ctx();
  if (!ctx) return fail(nullptr, LBM_ERR_OOM, "host allocation of the context failed");
  ctx->alloc = g_alloc;
  ctx->release = g_release;
  ctx->user = g_user;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(nullptr, e, "cudaGetDevice");
  }
  ctx->nx = nx; ctx->ny = ny; ctx->nz = nz;
  ctx->N = uint32_t(nx) * uint32_t(ny) * uint32_t(nz);
  ctx->tau = tau; ctx->rho0 = rho0; ctx->prec = prec; ctx->scheme = scheme;

  auto bail = [&](lbm_status s) {
    g_err = ctx->err;
    cudaStreamSynchronize(ctx->stream);
    ctx_free_all(ctx);
    delete ctx;
    return s;
  };
  const size_t pop_bytes = 19ull * ctx->N * storage_bytes(prec);
  for (int b = 0; b < (scheme == LBM_SCHEME_AA ? 1 : 2); ++b) {
    ctx->buf[b] = ctx_alloc(ctx, pop_bytes);
    if (!ctx->buf[b]) return bail(fail(ctx, LBM_ERR_OOM, "allocation of %zu bytes for populations failed", pop_bytes));
  }
  if (scheme == LBM_SCHEME_AA) ctx->buf[1] = ctx->buf[0];
  ctx->dred = static_cast<double*>(ctx_alloc(ctx, 4 * sizeof(double)));
  if (!ctx->dred) return bail(fail(ctx, LBM_ERR_OOM, "allocation of the reduction result failed"));
  ctx->derr = static_cast<uint32_t*>(ctx_alloc(ctx, sizeof(uint32_t)));
  if (!ctx->derr) return bail(fail(ctx, LBM_ERR_OOM, "allocation of the error word failed"));
  e = cudaMemsetAsync(ctx->derr, 0, sizeof(uint32_t), ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "clearing the error word"));

  lbm::SweepArgs& a = ctx->args;
  a.nx = nx; a.ny = ny; a.nz = nz; a.N = ctx->N;
  a.err = ctx->derr;
  a.div_nx = lbm::make_fastdiv(uint32_t(nx));
  a.div_ny = lbm::make_fastdiv(uint32_t(ny));
  a.div_nxh = lbm::make_fastdiv(uint32_t(nx / 2 > 0 ? nx / 2 : 1));
  a.periodic = 0;
  for (int ax = 0; ax < 3; ++ax)
    if (faces[2 * ax].kind == LBM_FACE_PERIODIC) a.periodic |= 1u << ax;
  a.rho0 = rho0;
  a.omega = 1.0 / tau;
  a.rho0f = float(rho0);
  a.omegaf = float(1.0 / tau);
  // 3 omega w_i of the BGK update's momentum term for the float sweep, as hi + lo
  // floats of omegaf / 6 (axis) and omegaf / 12 (diagonal): with a single rounded
  // constant every collision would gain or lose ~1e-7 of the node's momentum
  for (int c = 0; c < 2; ++c) {
    const double v = double(a.omegaf) / (c == 0 ? 6.0 : 12.0);
    a.mom_coef[c][0] = float(v);
    a.mom_coef[c][1] = float(v - double(a.mom_coef[c][0]));
  }
  const double zero[3] = {0.0, 0.0, 0.0};
  a.pressure = 0;
  for (int f = 0; f < 6; ++f) {
    const bool open = faces[f].kind != LBM_FACE_PERIODIC;
    const bool pres = faces[f].kind == LBM_FACE_PRESSURE;
    if (pres) a.pressure |= 1u << f;
    a.face[f].tab = nullptr;
    a.face[f].uni = face_node(f, open ? faces[f].u : zero, pres, pres ? faces[f].rho : 0.0);
    const bool per_node = open && (faces[f].u_table || (pres && faces[f].rho_table));
    if (per_node) {
      const size_t m = size_t(face_n1(f, nx, ny)) * face_n2(f, ny, nz);
      std::vector<lbm::FaceNode> host(m);
      for (size_t i = 0; i < m; ++i) {
        const double* u = faces[f].u_table ? faces[f].u_table + 3 * i : faces[f].u;
        const double r = pres ? (faces[f].rho_table ? faces[f].rho_table[i] : faces[f].rho) : 0.0;
        host[i] = face_node(f, u, pres, r);
      }
      const size_t bytes = m * sizeof(lbm::FaceNode);
      void* t = ctx_alloc(ctx, bytes);
      if (!t) return bail(fail(ctx, LBM_ERR_OOM, "allocation of face table %d failed", f));
      e = cudaMemcpy(t, host.data(), bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "copying a face table"));
      a.face[f].tab = static_cast<const lbm::FaceNode*>(t);
    }
  }
  e = dispatch_init(ctx, ctx->buf[0]);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "initial-state launch"));
  ctx->launches += 1;
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "initial state"));
  ctx->cur = 0;
  *out = ctx;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* ctx) {
  if (!ctx) return LBM_OK;
  DeviceGuard g(ctx->device);
  if (ctx->batch) lbm_batch_detach(ctx->batch, ctx->batch_slot);
  cudaStreamSynchronize(ctx->stream);
  ctx_free_all(ctx);
  delete ctx;
  return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx* ctx, void* cuda_stream) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int n) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0 (got %d)", n);
  if (ctx->scheme == LBM_SCHEME_AA && n % 2 != 0)
    return fail(ctx, LBM_ERR_ARG, "an AA lattice advances in pairs of steps (got n = %d)", n);
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  for (int i = 0; i < n; ++i) {
    set_direction(ctx, ctx->cur);
    LBM_CUDA(ctx, dispatch_sweep(ctx, false), "sweep launch");
    if (ctx->scheme == LBM_SCHEME_AB) ctx->cur ^= 1;
    ctx->steps += 1;
    ctx->launches += 1;
  }
  return LBM_OK;
}

lbm_status lbm_step_residual(lbm_ctx* ctx, int n, double* residual, double* mass) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (n < 1) return fail(ctx, LBM_ERR_ARG, "n must be >= 1 (got %d)", n);
  if (ctx->scheme == LBM_SCHEME_AA && n % 2 != 0)
    return fail(ctx, LBM_ERR_ARG, "an AA lattice advances in pairs of steps (got n = %d)", n);
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  if (lbm_status st0 = require_observable(ctx); st0 != LBM_OK) return st0;
  lbm_status st = ensure_reduction_buffers(ctx);
  if (st != LBM_OK) return st;
  // the n - 1 plain steps (an odd count for AA: issue them one by one)
  for (int i = 0; i < n - 1; ++i) {
    set_direction(ctx, ctx->cur);
    LBM_CUDA(ctx, dispatch_sweep(ctx, false), "sweep launch");
    if (ctx->scheme == LBM_SCHEME_AB) ctx->cur ^= 1;
    ctx->steps += 1;
    ctx->launches += 1;
  }
  set_direction(ctx, ctx->cur);
  LBM_CUDA(ctx, dispatch_sweep(ctx, true), "residual sweep launch");
  if (ctx->scheme == LBM_SCHEME_AB) ctx->cur ^= 1;
  ctx->steps += 1;
  ctx->launches += 1;
  return finish_reduction(ctx, residual, mass);
}

lbm_status lbm_residual(lbm_ctx* ctx, double* residual, double* mass) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  if (lbm_status st0 = require_observable(ctx); st0 != LBM_OK) return st0;
  lbm_status st = ensure_reduction_buffers(ctx);
  if (st != LBM_OK) return st;
  const bool sw = ctx->scheme == LBM_SCHEME_AA;
  cudaError_t e;
  switch (ctx->prec) {
    case LBM_F64: e = lbm::launch_state_reduce<double>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, ctx->snap, ctx->partials, sw, ctx->stream); break;
    case LBM_F32: e = lbm::launch_state_reduce<float>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, ctx->snap, ctx->partials, sw, ctx->stream); break;
    default: e = lbm::launch_state_reduce<__half>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, ctx->snap, ctx->partials, sw, ctx->stream); break;
  }
  LBM_CUDA(ctx, e, "state reduction launch");
  ctx->launches += 1;
  return finish_reduction(ctx, residual, mass);
}

lbm_status lbm_macros(lbm_ctx* ctx, void* rho, void* u) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (!rho && !u) return LBM_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  if (lbm_status st0 = require_observable(ctx); st0 != LBM_OK) return st0;
  const bool sw = ctx->scheme == LBM_SCHEME_AA;
  cudaError_t e;
  switch (ctx->prec) {
    case LBM_F64: e = lbm::launch_macros<double>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, rho, u, sw, ctx->stream); break;
    case LBM_F32: e = lbm::launch_macros<float>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, rho, u, sw, ctx->stream); break;
    default: e = lbm::launch_macros<__half>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, rho, u, sw, ctx->stream); break;
  }
  LBM_CUDA(ctx, e, "macros launch");
  ctx->launches += 1;
  return LBM_OK;
}

static lbm_status copy_populations(lbm_ctx* ctx, void* host_or_dev, int z0, int nzs, lbm_memory where, bool to_ctx) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (!host_or_dev) return fail(ctx, LBM_ERR_ARG, "buffer is NULL");
  if (z0 < 0 || nzs < 0 || z0 + nzs > ctx->nz) return fail(ctx, LBM_ERR_ARG, "planes %d..%d outside 0..%d", z0, z0 + nzs - 1, ctx->nz - 1);
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(ctx, LBM_ERR_ARG, "unknown memory kind %d", int(where));
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  if (lbm_status st0 = require_observable(ctx); st0 != LBM_OK) return st0;
  const size_t es = storage_bytes(ctx->prec);
  const size_t plane = size_t(ctx->nx) * ctx->ny;
  const size_t slab = plane * nzs * es;
  char* lat = static_cast<char*>(ctx->buf[ctx->cur]);
  char* user = static_cast<char*>(host_or_dev);
  cudaMemcpyKind kind = to_ctx ? (where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice)
                               : (where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  for (int k = 0; k < 19; ++k) {
    // an AA lattice keeps population k in slot -k between step pairs
    const int slot = ctx->scheme == LBM_SCHEME_AA ? lbm::opp(k) : k;
    char* l = lat + (size_t(slot) * ctx->N + size_t(z0) * plane) * es;
    char* u = user + size_t(k) * slab;
    LBM_CUDA(ctx, cudaMemcpyAsync(to_ctx ? l : u, to_ctx ? u : l, slab, kind, ctx->stream), "population copy");
  }
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "synchronising the population copy");
  return to_ctx ? LBM_OK : check_device_error(ctx);
}

lbm_status lbm_set_populations(lbm_ctx* ctx, const void* src, int z0, int nzs, lbm_memory where) {
  return copy_populations(ctx, const_cast<void*>(src), z0, nzs, where, true);
}

lbm_status lbm_get_populations(lbm_ctx* ctx, void* dst, int z0, int nzs, lbm_memory where) {
  return copy_populations(ctx, dst, z0, nzs, where, false);
}

}  // extern "C"

// Populations the on-site rule of a node code overwrites (bit k: population k), or 0
// for a value that is not a code. The codes name the normal by a lattice-vector index
// (include/lbm.h): planes 1..6, concave edges 7..18, convex edges -7..-18, corners
// 19..26, convex-edge/plane junctions 27..50.
static uint32_t rule_unknowns(int code) {
  auto dot = [](int k, const int* v) { return lbm::cx(k) * v[0] + lbm::cy(k) * v[1] + lbm::cz(k) * v[2]; };
  auto vec = [](int k, int* v) { v[0] = lbm::cx(k); v[1] = lbm::cy(k); v[2] = lbm::cz(k); };
  uint32_t m = 0;
  const int ac = code < 0 ? -code : code;
  if (code >= 1 && code <= 6) {
    int n[3];
    vec(code - 1, n);
    for (int k = 0; k < 19; ++k)
      if (dot(k, n) > 0) m |= 1u << k;
  } else if (ac >= 7 && ac <= 18) {
    int d[3];
    vec(ac - 1, d);
    for (int k = 0; k < 19; ++k) {
      if (code > 0) {
        // concave: from beyond either plane (normals = the axis parts of d)
        const bool b = (d[0] && lbm::cx(k) * d[0] > 0) || (d[1] && lbm::cy(k) * d[1] > 0) ||
                       (d[2] && lbm::cz(k) * d[2] > 0);
        if (b) m |= 1u << k;
      } else if (lbm::cx(k) == d[0] && lbm::cy(k) == d[1] && lbm::cz(k) == d[2]) {
        m |= 1u << k;  // convex: only c = d comes from the solid quadrant
      }
    }
  } else if (code >= 19 && code <= 26) {
    const int b = code - 19;
    const int sx = (b & 1) ? -1 : 1, sy = (b & 2) ? -1 : 1, sz = (b & 4) ? -1 : 1;
    for (int k = 0; k < 19; ++k)
      if (lbm::cx(k) * sx > 0 || lbm::cy(k) * sy > 0 || lbm::cz(k) * sz > 0) m |= 1u << k;
  } else if (code >= 27 && code <= 50) {
    int n[3];
    vec((code - 27) / 4, n);
    const int kd = lbm::junction_diagonal((code - 27) / 4, (code - 27) % 4);
    for (int k = 0; k < 19; ++k)
      if (dot(k, n) > 0 || k == kd) m |= 1u << k;
  }
  return m;
}

extern "C" {

lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* solid, const int8_t* code) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (!solid && !code) return fail(ctx, LBM_ERR_ARG, "solid and code are both NULL");
  if (ctx->scheme != LBM_SCHEME_AB) return fail(ctx, LBM_ERR_ARG, "a geometry needs the A/B scheme");
  if (ctx->batch) return fail(ctx, LBM_ERR_STATE, "detach the context from its batch first");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  // Geometry word per node (lbm_internal.h): solid nodes are flagged; a node with a
  // code gets its rule and must be able to stream everything its rule leaves alone;
  // any other node takes mid-grid bounce-back from its solid neighbours. Sources
  // outside a walled axis stay unflagged on code-0 nodes (the box closure fills them).
  const int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz;
  const int dims[3] = {nx, ny, nz};
  const uint32_t per = ctx->args.periodic;
  std::vector<uint32_t> links(ctx->N, 0u);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const size_t node = (size_t(z) * ny + y) * nx + x;
        const bool is_solid = solid && solid[node];
        const int c = code ? code[node] : 0;
        uint32_t blocked = 0, from_solid = 0;
        for (int k = 0; k < 19; ++k) {
          int p[3] = {x - lbm::cx(k), y - lbm::cy(k), z - lbm::cz(k)};
          bool inside = true;
          for (int a = 0; a < 3; ++a) {
            if (p[a] < 0 || p[a] >= dims[a]) {
              if (!((per >> a) & 1u)) inside = false;
              p[a] = (p[a] % dims[a] + dims[a]) % dims[a];
            }
          }
          const bool s_solid = inside && solid && solid[(size_t(p[2]) * ny + p[1]) * nx + p[0]];
          if (s_solid) from_solid |= 1u << k;
          if (s_solid || !inside) blocked |= 1u << k;
        }
        if (c == 0) {
          links[node] = is_solid ? lbm::SOLID_NODE : from_solid;
          continue;
        }
        const uint32_t rule_mask = rule_unknowns(c);
        if (!rule_mask) return fail(ctx, LBM_ERR_ARG, "node (%d, %d, %d): %d is not a boundary code", x, y, z, c);
        if (is_solid) return fail(ctx, LBM_ERR_ARG, "node (%d, %d, %d) is solid and has code %d", x, y, z, c);
        if (blocked & ~rule_mask)
          return fail(ctx, LBM_ERR_ARG,
                      "node (%d, %d, %d): code %d leaves a population from a solid or outside node unset", x,
                      y, z, c);
        const uint32_t rule = c > 0 ? uint32_t(c) : uint32_t(44 - c);
        links[node] = rule << lbm::RULE_SHIFT;
      }
  if (!ctx->args.links) {
    void* d = ctx_alloc(ctx, sizeof(uint32_t) * ctx->N);
    if (!d) return fail(ctx, LBM_ERR_OOM, "allocation of the geometry words failed");
    ctx->args.links = static_cast<const uint32_t*>(d);
  }
  LBM_CUDA(ctx, cudaMemcpyAsync(const_cast<uint32_t*>(ctx->args.links), links.data(), sizeof(uint32_t) * ctx->N,
                                cudaMemcpyHostToDevice, ctx->stream), "uploading the geometry words");
  // solid nodes are carried unchanged from buffer to buffer: start both alike
  LBM_CUDA(ctx, cudaMemcpyAsync(ctx->buf[ctx->cur ^ 1], ctx->buf[ctx->cur], 19ull * ctx->N * storage_bytes(ctx->prec),
                                cudaMemcpyDeviceToDevice, ctx->stream), "copying the state");
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "synchronising");
  return LBM_OK;
}

lbm_status lbm_rule_unknowns(int code, uint32_t* mask) {
  if (!mask) return fail(nullptr, LBM_ERR_ARG, "mask is NULL");
  const uint32_t m = rule_unknowns(code);
  if (!m) return fail(nullptr, LBM_ERR_ARG, "%d is not a boundary code", code);
  *mask = m;
  return LBM_OK;
}

lbm_status lbm_set_solid(lbm_ctx* ctx, const uint8_t* solid) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (!solid) return fail(ctx, LBM_ERR_ARG, "solid is NULL");
  return lbm_set_geometry(ctx, solid, nullptr);
}

lbm_status lbm_set_body_force(lbm_ctx* ctx, const double force[3]) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (!force) return fail(ctx, LBM_ERR_ARG, "force is NULL");
  if (!std::isfinite(force[0]) || !std::isfinite(force[1]) || !std::isfinite(force[2]))
    return fail(ctx, LBM_ERR_ARG, "force is not finite");
  if (ctx->scheme != LBM_SCHEME_AB) return fail(ctx, LBM_ERR_ARG, "a body force needs the A/B scheme");
  if (ctx->batch) return fail(ctx, LBM_ERR_STATE, "detach the context from its batch first");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  lbm::SweepArgs& a = ctx->args;
  const double tau = 1.0 / a.omega;
  for (int i = 0; i < 3; ++i) {
    a.force[i] = force[i];
    a.tforce[i] = tau * force[i];
    a.forcef[i] = float(force[i]);
    a.tforcef[i] = float(a.tforce[i]);
  }
  a.forced = (force[0] != 0.0 || force[1] != 0.0 || force[2] != 0.0) ? 1u : 0u;
  return LBM_OK;
}

lbm_status lbm_check_guards(lbm_ctx* ctx) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  if (lbm_status st0 = settle(ctx); st0 != LBM_OK) return st0;
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "synchronising");
  std::vector<unsigned char> h(2 * GUARD);
  for (size_t i = 0; i < ctx->allocations.size(); ++i) {
    const Allocation& a = ctx->allocations[i];
    const char* base = static_cast<const char*>(a.ptr);
    LBM_CUDA(ctx, cudaMemcpy(h.data(), base, GUARD, cudaMemcpyDeviceToHost), "reading a guard");
    LBM_CUDA(ctx, cudaMemcpy(h.data() + GUARD, base + GUARD + a.bytes, GUARD, cudaMemcpyDeviceToHost),
             "reading a guard");
    for (size_t j = 0; j < 2 * GUARD; ++j)
      if (h[j] != GUARD_BYTE)
        return fail(ctx, LBM_ERR_STATE, "buffer %zu (%zu bytes): guard %s it overwritten at byte %zu", i, a.bytes,
                    j < GUARD ? "below" : "above", j < GUARD ? j : j - GUARD);
  }
  return LBM_OK;
}

lbm_status lbm_debug_bounds_errors(int* enabled, uint64_t* count) {
  if (!enabled || !count) return fail(nullptr, LBM_ERR_ARG, "enabled or count is NULL");
#ifdef LBM_DEBUG_BOUNDS
  *enabled = 1;
#else
  *enabled = 0;
#endif
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, LBM_ERR_CUDA, "device synchronisation failed");
  }
  const uint32_t c[3] = {lbm::bounds_errors<double>(), lbm::bounds_errors<float>(), lbm::bounds_errors<__half>()};
  uint64_t total = 0;
  for (uint32_t v : c) {
    if (v == ~0u) return fail(nullptr, LBM_ERR_CUDA, "reading the bounds-error words failed");
    total += v;
  }
  *count = total;
  return LBM_OK;
}

lbm_status lbm_debug_drop_staged_copies(lbm_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  ctx->args.drop_copies = enable ? 1u : 0u;
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* ctx) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronisation");
  LBM_CUDA(ctx, cudaGetLastError(), "pending error");
  return check_device_error(ctx);
}

lbm_status lbm_info(const lbm_ctx* ctx, lbm_info_t* out) {
  if (!ctx || !out) return fail(nullptr, LBM_ERR_ARG, "ctx or out is NULL");
  out->nx = ctx->nx;
  out->ny = ctx->ny;
  out->nz = ctx->nz;
  out->precision = ctx->prec;
  out->steps = ctx->steps;
  out->kernel_launches = ctx->launches;
  out->bytes_per_update = int64_t(38 * storage_bytes(ctx->prec));
  out->device_bytes = ctx->device_bytes;
  out->scheme = ctx->scheme;
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Batches: many resident lattices advanced by one persistent launch per step.
// ---------------------------------------------------------------------------------

static lbm_status bfail(lbm_batch* b, lbm_status st, const char* msg) {
  if (b) b->err = msg;
  g_err = msg;
  return st;
}

static lbm_status bcuda(lbm_batch* b, cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, buf);
}

#define LBM_BCUDA(b, expr, what)                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return bcuda(b, e_, what); \
  } while (0)

static void* batch_alloc(lbm_batch* b, size_t bytes) {
  void* p = nullptr;
  if (b->alloc) {
    p = b->alloc(bytes, b->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    b->allocations.push_back({p, bytes});
    b->device_bytes += int64_t(bytes);
  }
  return p;
}

static void batch_release(lbm_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  for (lbm_ctx* c : b->slots)
    if (c) {
      c->batch = nullptr;
      c->batch_slot = -1;
    }
  for (auto it = b->allocations.rbegin(); it != b->allocations.rend(); ++it) {
    if (b->release) b->release(it->ptr, b->user);
    else cudaFree(it->ptr);
  }
  b->allocations.clear();
  if (b->h_hdr) cudaFreeHost(b->h_hdr);
  if (b->h_ent) cudaFreeHost(b->h_ent);
  if (b->h_res) cudaFreeHost(b->h_res);
  if (b->h_chunks) cudaFreeHost(b->h_chunks);
  if (b->table_free) cudaEventDestroy(b->table_free);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// Step i of a batched n-step loop: A/B lattices alternate the buffer direction with
// the parity; AA lattices (all at a step-pair boundary when a loop starts) alternate
// the gather-scatter and in-place steps.
// Every launch starts with its chunk counter at zero (a memset in stream order, so a
// captured step loop holds one memset node before each sweep node).
static cudaError_t batch_launch_sweep(lbm_batch* b, uint32_t parity, bool resid) {
  const int mode = b->scheme == LBM_SCHEME_AA ? (parity ? 2 : 1) : 0;
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(uint32_t), b->stream);
  if (e != cudaSuccess) return e;
  const int grid = b->grid;
  switch (b->prec) {
    case LBM_F64:
      return lbm::launch_sweep_batched<double>(b->d_hdr, b->d_ent, b->d_chunks, b->d_next, parity, resid, mode,
                                               grid, b->stream);
    case LBM_F32:
      return lbm::launch_sweep_batched<float>(b->d_hdr, b->d_ent, b->d_chunks, b->d_next, parity, resid, mode,
                                              grid, b->stream);
    default:
      return lbm::launch_sweep_batched<__half>(b->d_hdr, b->d_ent, b->d_chunks, b->d_next, parity, resid, mode,
                                               grid, b->stream);
  }
}

// Rows of the chunk table (without its sentinel).
constexpr uint32_t kMaxChunks = 65535;

// Guided self-scheduling of the batch's global block range over `grid` CTAs: each chunk
// takes 1 / (2 grid) of the blocks still unassigned (at least `min_chunk`), so the first
// draws are large (few descriptor changes) and the last are single blocks (the CTAs
// end together). Writes rows 0..n-1 and the sentinel row n; returns n, or 0 if the
// table would need more than kMaxChunks rows.
static uint32_t build_chunks(const lbm::BatchEntry* ents, uint32_t nent, uint32_t total, uint32_t grid,
                             uint32_t min_chunk, lbm::BatchChunk* out) {
  uint32_t n = 0, pos = 0, e = 0;
  const uint64_t div = 2ull * (grid ? grid : 1);
  while (pos < total) {
    if (n >= kMaxChunks) return 0;
    const uint32_t rem = total - pos;
    uint32_t size = uint32_t((rem + div - 1) / div);
    if (size < min_chunk) size = min_chunk;
    if (size > rem) size = rem;
    while (ents[e].block_begin + ents[e].nblocks <= pos) ++e;
    out[n++] = {pos, e};
    pos += size;
  }
  out[n] = {total, nent};
  return n;
}

// Issue n batched steps (the last with the residual reductions when `resid`).
static cudaError_t batch_issue(lbm_batch* b, int n, bool resid) {
  for (int i = 0; i < n; ++i) {
    cudaError_t e = batch_launch_sweep(b, uint32_t(i & 1), resid && i == n - 1);
    if (e != cudaSuccess) return e;
  }
  if (resid) return lbm::launch_batch_final_reduce(b->d_hdr, b->d_ent, b->capacity, b->d_res, b->stream);
  return cudaSuccess;
}

extern "C" {

lbm_status lbm_batch_create(int capacity, lbm_precision prec, lbm_batch** out) {
  if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (capacity < 1 || capacity > (1 << 20)) return bfail(nullptr, LBM_ERR_ARG, "capacity must be in 1 .. 2^20");
  if (prec < LBM_F64 || prec > LBM_F16_SHIFTED) return bfail(nullptr, LBM_ERR_ARG, "unknown precision");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(nullptr, LBM_ERR_OOM, "host allocation of the batch failed");
  b->capacity = capacity;
  b->prec = prec;
  b->alloc = g_alloc;
  b->release = g_release;
  b->user = g_user;
  auto bail = [&](lbm_status st) {
    batch_release(b);
    delete b;
    return st;
  };
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) return bail(bcuda(nullptr, e, "cudaGetDevice"));
  b->slots.assign(capacity, nullptr);
  b->has_result.assign(capacity, 0);
  e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(bcuda(nullptr, e, "creating the batch stream"));
  b->own_stream = true;
  e = cudaEventCreateWithFlags(&b->table_free, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(bcuda(nullptr, e, "creating the table event"));
  const size_t ent_bytes = sizeof(lbm::BatchEntry) * size_t(capacity);
  const size_t res_bytes = 4 * sizeof(double) * size_t(capacity);
  const size_t chunk_bytes = sizeof(lbm::BatchChunk) * (size_t(kMaxChunks) + 1);
  if ((e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_hdr), sizeof(lbm::BatchHeader), cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_ent), ent_bytes, cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_res), res_bytes, cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_chunks), chunk_bytes, cudaHostAllocDefault)) != cudaSuccess)
    return bail(bcuda(nullptr, e, "pinned host table"));
  b->d_hdr = static_cast<lbm::BatchHeader*>(batch_alloc(b, sizeof(lbm::BatchHeader)));
  b->d_ent = static_cast<lbm::BatchEntry*>(batch_alloc(b, ent_bytes));
  b->d_res = static_cast<double*>(batch_alloc(b, res_bytes));
  b->d_chunks = static_cast<lbm::BatchChunk*>(batch_alloc(b, chunk_bytes));
  b->d_next = static_cast<uint32_t*>(batch_alloc(b, 256));
  if (!b->d_hdr || !b->d_ent || !b->d_res || !b->d_chunks || !b->d_next)
    return bail(bfail(nullptr, LBM_ERR_OOM, "device allocation of the batch table failed"));
  memset(b->h_hdr, 0, sizeof(lbm::BatchHeader));
  e = cudaMemcpy(b->d_hdr, b->h_hdr, sizeof(lbm::BatchHeader), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(bcuda(nullptr, e, "clearing the batch table"));
  // one grid for every batched variant: SMs x the smallest residency among them (a grid
  // of the A/B step's own, larger residency measured 1 - 2 % slower on a serving mix)
  b->grid = 0;
  for (int r = 0; r < 2; ++r)
    for (int m = 0; m < 3; ++m) {
      int g = 0;
      switch (prec) {
        case LBM_F64: g = lbm::batched_grid<double>(r != 0, m); break;
        case LBM_F32: g = lbm::batched_grid<float>(r != 0, m); break;
        default: g = lbm::batched_grid<__half>(r != 0, m); break;
      }
      if (g <= 0) return bail(bfail(nullptr, LBM_ERR_CUDA, "occupancy query for the batched sweep failed"));
      b->grid = (b->grid == 0 || g < b->grid) ? g : b->grid;
    }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  DeviceGuard g(b->device);
  batch_release(b);
  delete b;
  return LBM_OK;
}

lbm_status lbm_batch_set_stream(lbm_batch* b, void* cuda_stream) {
  if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
  DeviceGuard g(b->device);
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "synchronising the previous stream");
  for (auto& gr : b->graphs) cudaGraphExecDestroy(gr.exec);
  b->graphs.clear();
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = false;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  return LBM_OK;
}

lbm_status lbm_batch_attach(lbm_batch* b, int slot, lbm_ctx* ctx) {
  if (!b || !ctx) return bfail(b, LBM_ERR_ARG, "batch or ctx is NULL");
  if (slot < 0 || slot >= b->capacity) return bfail(b, LBM_ERR_ARG, "slot out of range");
  if (b->slots[slot]) return bfail(b, LBM_ERR_STATE, "slot is occupied");
  if (ctx->batch) return bfail(b, LBM_ERR_STATE, "context is attached to a batch already");
  if (ctx->prec != b->prec) return bfail(b, LBM_ERR_ARG, "context precision differs from the batch's");
  if (ctx->device != b->device) return bfail(b, LBM_ERR_ARG, "context lives on another device");
  int attached = 0;
  for (lbm_ctx* c : b->slots) attached += c ? 1 : 0;
  if (attached > 0 && int(ctx->scheme) != b->scheme)
    return bfail(b, LBM_ERR_ARG, "context streaming scheme differs from the batch's");
  if (ctx->scheme == LBM_SCHEME_AA && ctx->steps % 2 != 0)
    return bfail(b, LBM_ERR_STATE, "an AA context joins a batch between step pairs only");
  DeviceGuard g(b->device);
  lbm_status st = ensure_reduction_buffers(ctx);
  if (st != LBM_OK) return bfail(b, st, ctx->err.c_str());
  LBM_BCUDA(b, cudaStreamSynchronize(ctx->stream), "waiting for the context's own work");
  b->slots[slot] = ctx;
  b->has_result[slot] = 0;
  b->scheme = int(ctx->scheme);
  ctx->batch = b;
  ctx->batch_slot = slot;
  return LBM_OK;
}

lbm_status lbm_batch_detach(lbm_batch* b, int slot) {
  if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
  if (slot < 0 || slot >= b->capacity) return bfail(b, LBM_ERR_ARG, "slot out of range");
  lbm_ctx* ctx = b->slots[slot];
  if (!ctx) return LBM_OK;
  DeviceGuard g(b->device);
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "waiting for the batch");
  b->slots[slot] = nullptr;
  b->has_result[slot] = 0;
  ctx->batch = nullptr;
  ctx->batch_slot = -1;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n, int residual) {
  if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
  if (n < 1) return bfail(b, LBM_ERR_ARG, "n must be >= 1");
  if (b->scheme == LBM_SCHEME_AA && n % 2 != 0) return bfail(b, LBM_ERR_ARG, "a batch of AA lattices steps in pairs");
  DeviceGuard g(b->device);
  // the previous upload must have read the host mirror before it is rewritten
  LBM_BCUDA(b, cudaEventSynchronize(b->table_free), "waiting for the previous table upload");
  uint32_t nent = 0, blocks = 0;
  for (int slot = 0; slot < b->capacity; ++slot) {
    lbm_ctx* c = b->slots[slot];
    if (!c) continue;
    lbm::BatchEntry& e = b->h_ent[nent++];
    e.a = c->args;
    e.buf[0] = c->buf[0];
    e.buf[1] = c->buf[1];
    e.cur = uint32_t(c->cur);
    e.block_begin = blocks;
    e.nblocks = lbm::sweep_blocks(c->N);
    e.slot = uint32_t(slot);
    blocks += e.nblocks;
  }
  b->h_hdr->nentries = nent;
  b->h_hdr->total_blocks = blocks;
  b->total_blocks = blocks;
  if (nent == 0) return LBM_OK;
  uint32_t nchunks = 0;
  for (uint32_t min_chunk = 1; nchunks == 0; min_chunk *= 2)
    nchunks = build_chunks(b->h_ent, nent, blocks, uint32_t(b->grid), min_chunk, b->h_chunks);
  b->h_hdr->nchunks = nchunks;
  const bool resid = residual != 0;
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(lbm::BatchHeader), cudaMemcpyHostToDevice, b->stream),
            "uploading the batch header");
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_ent, b->h_ent, sizeof(lbm::BatchEntry) * nent, cudaMemcpyHostToDevice, b->stream),
            "uploading the batch table");
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_chunks, b->h_chunks, sizeof(lbm::BatchChunk) * (nchunks + 1),
                               cudaMemcpyHostToDevice, b->stream),
            "uploading the chunk table");
  LBM_BCUDA(b, cudaEventRecord(b->table_free, b->stream), "recording the table event");
  if (b->stream) {
    // the n-step loop as one CUDA graph; its kernels read the table from device memory,
    // so one graph per (n, residual) serves every membership of the batch
    cudaGraphExec_t exec = nullptr;
    for (auto& gr : b->graphs)
      if (gr.n == n && gr.resid == resid && gr.scheme == b->scheme) exec = gr.exec;
    if (!exec) {
      cudaGraph_t graph = nullptr;
      LBM_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "beginning graph capture");
      cudaError_t e = batch_issue(b, n, resid);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
      if (e != cudaSuccess) return bcuda(b, e, "capturing the batched steps");
      if (e2 != cudaSuccess) return bcuda(b, e2, "ending graph capture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return bcuda(b, e, "instantiating the step graph");
      if (b->graphs.size() >= 8) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        b->graphs.erase(b->graphs.begin());
      }
      b->graphs.push_back({n, resid, b->scheme, exec});
    }
    LBM_BCUDA(b, cudaGraphLaunch(exec, b->stream), "launching the step graph");
  } else {
    LBM_BCUDA(b, batch_issue(b, n, resid), "batched step launch");
  }
  if (resid)
    LBM_BCUDA(b, cudaMemcpyAsync(b->h_res, b->d_res, 4 * sizeof(double) * b->capacity, cudaMemcpyDeviceToHost, b->stream),
              "reading the batch results");
  b->results_valid = resid;
  for (int slot = 0; slot < b->capacity; ++slot) {
    lbm_ctx* c = b->slots[slot];
    b->has_result[slot] = (c && resid) ? 1 : 0;
    if (!c) continue;
    if (c->scheme == LBM_SCHEME_AB) c->cur ^= (n & 1);
    c->steps += n;
  }
  b->steps += n;
  b->launches += n + (resid ? 1 : 0);
  return LBM_OK;
}

lbm_status lbm_batch_results(lbm_batch* b, double* residual, double* mass, int* status) {
  if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
  DeviceGuard g(b->device);
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "waiting for the batch");
  for (int slot = 0; slot < b->capacity; ++slot) {
    double r = NAN, m = NAN;
    int st = 1;  // no result for this slot
    if (b->results_valid && b->has_result[slot]) {
      const double* h = b->h_res + 4 * slot;
      r = h[2] > 0.0 ? std::sqrt(h[1]) / std::sqrt(h[2]) : std::sqrt(h[1]);
      m = h[0];
      st = (h[3] != 0.0 || !std::isfinite(h[0]) || !std::isfinite(r)) ? int(LBM_ERR_DIVERGED) : int(LBM_OK);
    }
    if (residual) residual[slot] = r;
    if (mass) mass[slot] = m;
    if (status) status[slot] = st;
  }
  return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch* b, lbm_batch_info_t* out) {
  if (!b || !out) return bfail(nullptr, LBM_ERR_ARG, "batch or out is NULL");
  int attached = 0;
  int64_t nodes = 0;
  for (lbm_ctx* c : b->slots)
    if (c) {
      ++attached;
      nodes += c->N;
    }
  out->capacity = b->capacity;
  out->attached = attached;
  out->grid = b->grid;
  out->nodes = nodes;
  out->steps = b->steps;
  out->kernel_launches = b->launches;
  out->device_bytes = b->device_bytes;
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_err.c_str(); }

}  // extern "C"

extern "C" {

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

}  // extern "C"
