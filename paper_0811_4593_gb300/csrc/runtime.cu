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
#include "lbm_internal.h"

namespace {

lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_release = nullptr;
void* g_user = nullptr;
thread_local std::string g_err = "no error";

struct Allocation {
  void* ptr;
  size_t bytes;
};

}  // namespace

struct lbm_ctx {
  int device = 0;
  int nx = 0, ny = 0, nz = 0;
  uint32_t N = 0;
  double tau = 1.0, rho0 = 1.0;
  lbm_precision prec = LBM_F32;
  lbm::SweepArgs args{};
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;  // buf[cur] holds the current post-collision state
  void* snap = nullptr;
  double* partials = nullptr;
  double* dred = nullptr;
  cudaStream_t stream = nullptr;
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
  if (ctx->alloc) {
    p = ctx->alloc(bytes, ctx->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    ctx->allocations.push_back({p, bytes});
    ctx->device_bytes += int64_t(bytes);
  }
  return p;
}

void ctx_free_all(lbm_ctx* ctx) {
  for (auto it = ctx->allocations.rbegin(); it != ctx->allocations.rend(); ++it) {
    if (ctx->release) ctx->release(it->ptr, ctx->user);
    else cudaFree(it->ptr);
  }
  ctx->allocations.clear();
  ctx->device_bytes = 0;
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
  for (int a = 0; a < 3; ++a) {
    const int k0 = faces[2 * a].kind, k1 = faces[2 * a + 1].kind;
    for (int k : {k0, k1})
      if (k != LBM_FACE_PERIODIC && k != LBM_FACE_VELOCITY) return fail(nullptr, LBM_ERR_ARG, "axis %d: unknown face kind %d", a, k);
    if ((k0 == LBM_FACE_PERIODIC) != (k1 == LBM_FACE_PERIODIC))
      return fail(nullptr, LBM_ERR_ARG, "axis %d: periodic faces must come in pairs", a);
  }
  for (int f = 0; f < 6; ++f) {
    if (faces[f].kind != LBM_FACE_VELOCITY) continue;
    const int a = f / 2;
    const double sg = (f % 2 == 0) ? 1.0 : -1.0;
    if (faces[f].u_table) {
      const size_t m = size_t(face_n1(f, nx, ny)) * face_n2(f, ny, nz);
      for (size_t i = 0; i < m; ++i) {
        const double* u = faces[f].u_table + 3 * i;
        if (!std::isfinite(u[0]) || !std::isfinite(u[1]) || !std::isfinite(u[2]))
          return fail(nullptr, LBM_ERR_ARG, "face %d: non-finite velocity at table entry %zu", f, i);
        if (!(std::fabs(sg * u[a]) < 1.0)) return fail(nullptr, LBM_ERR_ARG, "face %d: |u.n| >= 1 at table entry %zu", f, i);
      }
    } else {
      const double* u = faces[f].u;
      if (!std::isfinite(u[0]) || !std::isfinite(u[1]) || !std::isfinite(u[2]))
        return fail(nullptr, LBM_ERR_ARG, "face %d: non-finite velocity", f);
      if (!(std::fabs(u[a]) < 1.0)) return fail(nullptr, LBM_ERR_ARG, "face %d: |u.n| >= 1", f);
    }
  }
  return LBM_OK;
}

cudaError_t dispatch_sweep(lbm_ctx* ctx, bool resid) {
  switch (ctx->prec) {
    case LBM_F64: return lbm::launch_sweep<double>(ctx->args, resid, ctx->stream);
    case LBM_F32: return lbm::launch_sweep<float>(ctx->args, resid, ctx->stream);
    default: return lbm::launch_sweep<__half>(ctx->args, resid, ctx->stream);
  }
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

// Final fold of the partial sums and the host-side residual.
lbm_status finish_reduction(lbm_ctx* ctx, double* residual, double* mass) {
  LBM_CUDA(ctx, lbm::launch_final_reduce(ctx->partials, lbm::sweep_blocks(ctx->N), ctx->dred, ctx->stream),
           "final reduction launch");
  ctx->launches += 1;
  double h[4];
  LBM_CUDA(ctx, cudaMemcpyAsync(h, ctx->dred, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "reading reductions");
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "synchronising after reductions");
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
  if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
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
  ctx->tau = tau; ctx->rho0 = rho0; ctx->prec = prec;

  auto bail = [&](lbm_status s) {
    g_err = ctx->err;
    cudaStreamSynchronize(ctx->stream);
    ctx_free_all(ctx);
    delete ctx;
    return s;
  };
  const size_t pop_bytes = 19ull * ctx->N * storage_bytes(prec);
  for (int b = 0; b < 2; ++b) {
    ctx->buf[b] = ctx_alloc(ctx, pop_bytes);
    if (!ctx->buf[b]) return bail(fail(ctx, LBM_ERR_OOM, "allocation of %zu bytes for populations failed", pop_bytes));
  }
  ctx->dred = static_cast<double*>(ctx_alloc(ctx, 4 * sizeof(double)));
  if (!ctx->dred) return bail(fail(ctx, LBM_ERR_OOM, "allocation of the reduction result failed"));

  lbm::SweepArgs& a = ctx->args;
  a.nx = nx; a.ny = ny; a.nz = nz; a.N = ctx->N;
  a.div_nx = lbm::make_fastdiv(uint32_t(nx));
  a.div_ny = lbm::make_fastdiv(uint32_t(ny));
  a.periodic = 0;
  for (int ax = 0; ax < 3; ++ax)
    if (faces[2 * ax].kind == LBM_FACE_PERIODIC) a.periodic |= 1u << ax;
  a.rho0 = rho0;
  a.omega = 1.0 / tau;
  for (int f = 0; f < 6; ++f) {
    a.face[f].tab = nullptr;
    for (int j = 0; j < 3; ++j) a.face[f].u[j] = faces[f].kind == LBM_FACE_VELOCITY ? faces[f].u[j] : 0.0;
    if (faces[f].kind == LBM_FACE_VELOCITY && faces[f].u_table) {
      const size_t bytes = 3ull * face_n1(f, nx, ny) * face_n2(f, ny, nz) * sizeof(double);
      void* t = ctx_alloc(ctx, bytes);
      if (!t) return bail(fail(ctx, LBM_ERR_OOM, "allocation of face table %d failed", f));
      e = cudaMemcpy(t, faces[f].u_table, bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "copying a face table"));
      a.face[f].tab = static_cast<const double*>(t);
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
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  for (int i = 0; i < n; ++i) {
    ctx->args.src = ctx->buf[ctx->cur];
    ctx->args.dst = ctx->buf[ctx->cur ^ 1];
    LBM_CUDA(ctx, dispatch_sweep(ctx, false), "sweep launch");
    ctx->cur ^= 1;
    ctx->steps += 1;
    ctx->launches += 1;
  }
  return LBM_OK;
}

lbm_status lbm_step_residual(lbm_ctx* ctx, int n, double* residual, double* mass) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  if (n < 1) return fail(ctx, LBM_ERR_ARG, "n must be >= 1 (got %d)", n);
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  lbm_status st = ensure_reduction_buffers(ctx);
  if (st != LBM_OK) return st;
  st = lbm_step(ctx, n - 1);
  if (st != LBM_OK) return st;
  ctx->args.src = ctx->buf[ctx->cur];
  ctx->args.dst = ctx->buf[ctx->cur ^ 1];
  LBM_CUDA(ctx, dispatch_sweep(ctx, true), "residual sweep launch");
  ctx->cur ^= 1;
  ctx->steps += 1;
  ctx->launches += 1;
  return finish_reduction(ctx, residual, mass);
}

lbm_status lbm_residual(lbm_ctx* ctx, double* residual, double* mass) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LBM_ERR_CUDA, "cannot make device %d current", ctx->device);
  lbm_status st = ensure_reduction_buffers(ctx);
  if (st != LBM_OK) return st;
  cudaError_t e;
  switch (ctx->prec) {
    case LBM_F64: e = lbm::launch_state_reduce<double>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, ctx->snap, ctx->partials, ctx->stream); break;
    case LBM_F32: e = lbm::launch_state_reduce<float>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, ctx->snap, ctx->partials, ctx->stream); break;
    default: e = lbm::launch_state_reduce<__half>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, ctx->snap, ctx->partials, ctx->stream); break;
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
  cudaError_t e;
  switch (ctx->prec) {
    case LBM_F64: e = lbm::launch_macros<double>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, rho, u, ctx->stream); break;
    case LBM_F32: e = lbm::launch_macros<float>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, rho, u, ctx->stream); break;
    default: e = lbm::launch_macros<__half>(ctx->buf[ctx->cur], ctx->N, ctx->rho0, rho, u, ctx->stream); break;
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
  const size_t es = storage_bytes(ctx->prec);
  const size_t plane = size_t(ctx->nx) * ctx->ny;
  const size_t slab = plane * nzs * es;
  char* lat = static_cast<char*>(ctx->buf[ctx->cur]);
  char* user = static_cast<char*>(host_or_dev);
  cudaMemcpyKind kind = to_ctx ? (where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice)
                               : (where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  for (int k = 0; k < 19; ++k) {
    char* l = lat + (size_t(k) * ctx->N + size_t(z0) * plane) * es;
    char* u = user + size_t(k) * slab;
    LBM_CUDA(ctx, cudaMemcpyAsync(to_ctx ? l : u, to_ctx ? u : l, slab, kind, ctx->stream), "population copy");
  }
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "synchronising the population copy");
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* ctx, const void* src, int z0, int nzs, lbm_memory where) {
  return copy_populations(ctx, const_cast<void*>(src), z0, nzs, where, true);
}

lbm_status lbm_get_populations(lbm_ctx* ctx, void* dst, int z0, int nzs, lbm_memory where) {
  return copy_populations(ctx, dst, z0, nzs, where, false);
}

lbm_status lbm_sync(lbm_ctx* ctx) {
  if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  LBM_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronisation");
  LBM_CUDA(ctx, cudaGetLastError(), "pending error");
  return LBM_OK;
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
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

}  // extern "C"
