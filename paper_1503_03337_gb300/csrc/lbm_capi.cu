// C-ABI of liblbm: handle lifecycle, parameter validation and the host
// orchestration of the single-domain kernels (declared in include/lbm.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

#include "lbm_internal.h"

using namespace lbm;

struct lbm_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  DomainDesc d{};
  lbm_geom geom{};
  lbm_params params{};
  int64_t n = 0;
  BlockShape block{32, 8, 1};
  // reductions
  double* u_prev = nullptr;     // 3*N snapshot, allocated on first use
  int have_prev = 0;
  int64_t prev_step = -1;
  int64_t stats_step = -1;      // step of the statistics in stats_host
  int64_t stats_prev_step = -1;
  double* partials = nullptr;   // kReduceBlocks * kNumStats
  double* stats_host = nullptr; // mapped pinned, kNumStats
  double* stats_dev = nullptr;  // device alias of stats_host
  void* staging = nullptr;      // grow-only device buffer for host transfers
  size_t staging_bytes = 0;
  int64_t bytes = 0;
  uint8_t* solid_bytes = nullptr;   // N bytes: the solid-node mask, or null
  uint32_t* solid_links = nullptr;  // N words: its link bits (d.solid)
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return LBM_ECUDA;
}

size_t storage_bytes(int storage) {
  switch (storage) {
    case LBM_STORAGE_F64: return 8;
    case LBM_STORAGE_F32: return 4;
    case LBM_STORAGE_F16:
    case LBM_STORAGE_BF16: return 2;
  }
  return 0;
}

// Makes the handle's device current for the scope.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

int apply_params(lbm_handle* h, const lbm_params* p) {
  double s[6] = {p->s_c, p->s_e, p->s_q, p->s_nu, p->s_pi, p->s_t};
  if (p->nu > 0.0) s[3] = 1.0 / (3.0 * p->nu + 0.5);
  if (!(std::isfinite(p->nu))) return fail(LBM_EINVAL, "nu is not finite");
  for (int k = 0; k < 6; ++k) {
    if (k == 4 && h->d.Q == 14) continue;  // s_pi exists only for Q18 and Q26
    if (!(s[k] > 0.0 && s[k] < 2.0))
      return fail(LBM_EINVAL, "relaxation rates must lie in (0, 2)");
  }
  if (!finite_all(p->force, 3) || !std::isfinite(p->force_period) ||
      !std::isfinite(p->p_ref))
    return fail(LBM_EINVAL, "force, period and p_ref must be finite");
  if (p->residual_interval < 0) return fail(LBM_EINVAL, "residual_interval < 0");
  if (p->rounding != LBM_ROUND_NEAREST && p->rounding != LBM_ROUND_STOCHASTIC)
    return fail(LBM_EINVAL, "unknown rounding mode");
  if (!finite_all(p->p_face, 6) || !finite_all(p->p_amp, 6) || !std::isfinite(p->p_period))
    return fail(LBM_EINVAL, "face pressures must be finite");
  if (h->d.Q == 14) s[4] = s[1];
  h->params = *p;
  for (int k = 0; k < 6; ++k) h->d.s[k] = s[k];
  for (int k = 0; k < 3; ++k) h->d.force[k] = p->force[k];
  h->d.period = p->force_period;
  h->d.p_ref = p->p_ref;
  h->d.rounding = p->rounding;
  for (int f = 0; f < 6; ++f) {
    h->d.p_face[f] = p->p_face[f];
    h->d.p_amp[f] = p->p_amp[f];
  }
  h->d.p_period = p->p_period;
  return LBM_OK;
}

int apply_geometry(lbm_handle* h, const lbm_geom* g) {
  if (h->solid_bytes)
    for (int f = 0; f < 6; ++f)
      if (g->face[f] == LBM_NEQ_VELOCITY || g->face[f] == LBM_NEQ_PRESSURE)
        return fail(LBM_EINVAL, "extrapolation faces do not combine with solid nodes");
  // set_faces changes the handle only once every check has passed
  DomainDesc d = h->d;
  if (const char* why = set_faces(d, g)) return fail(LBM_EINVAL, why);
  if (h->solid_bytes) {  // the link bits follow the faces' wraps and mirrors
    cudaError_t e = launch_solid_links(d, h->solid_bytes, h->solid_links, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "solid links");
  }
  h->d = d;
  h->geom = *g;
  return LBM_OK;
}

int check(lbm_handle* h) {
  if (!h) return fail(LBM_EINVAL, "null handle");
  return LBM_OK;
}

}  // namespace

void lbm::set_last_error(const std::string& msg) { g_last_error = msg; }

extern "C" {

const char* lbm_last_error(void) { return g_last_error.c_str(); }

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "non-finite values (unstable run)";
    case LBM_ETIMEOUT: return "device-side wait timed out";
    case LBM_EBUSY: return "busy (no free slot or memory budget)";
  }
  return "unknown error";
}

int lbm_create(const lbm_desc* desc, void* cuda_stream, lbm_handle** out) {
  if (!desc || !out) return fail(LBM_EINVAL, "null argument");
  *out = nullptr;
  if (desc->Q != 14 && desc->Q != 18 && desc->Q != 26)
    return fail(LBM_EINVAL, "Q must be 14, 18 or 26");
  if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1)
    return fail(LBM_EINVAL, "grid sizes must be >= 1");
  const size_t b = storage_bytes(desc->storage);
  if (!b) return fail(LBM_EINVAL, "unknown storage type");
  const int64_t N = (int64_t)desc->nx * desc->ny * desc->nz;
  // cell indices are 32-bit; population offsets a*N + i are 64-bit where
  // Q*N >= 2^31 (the step's wide kernels)
  if (N >= (int64_t(1) << 31) || desc->nz > 65535)
    return fail(LBM_EINVAL, "domain too large (nx*ny*nz must be < 2^31, nz <= 65535)");

  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return fail(LBM_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaGetDevice");
  }
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->d.Q = desc->Q;
  h->d.nx = desc->nx;
  h->d.ny = desc->ny;
  h->d.nz = desc->nz;
  h->d.storage = desc->storage;
  h->d.N = N;
  h->block = default_block(desc->nx, desc->ny);

  const size_t fbytes = (size_t)N * desc->Q * b;
  e = cudaMalloc(&h->d.f, fbytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(LBM_ENOMEM, "cudaMalloc of populations failed");
  }
  e = cudaMalloc(&h->partials, sizeof(double) * kReduceBlocks * kNumStats);
  if (e == cudaSuccess)
    e = cudaHostAlloc(&h->stats_host, sizeof(double) * kNumStats, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&h->stats_dev, h->stats_host, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    lbm_destroy(h);
    return fail(LBM_ENOMEM, "allocation of reduction workspace failed");
  }
  std::memset(h->stats_host, 0, sizeof(double) * kNumStats);
  h->bytes = (int64_t)fbytes + sizeof(double) * kReduceBlocks * kNumStats;
  e = cudaMemsetAsync(h->d.f, 0, fbytes, h->stream);
  if (e != cudaSuccess) {
    lbm_destroy(h);
    return cuda_fail(e, "cudaMemsetAsync");
  }

  lbm_geom g{};
  for (int f = 0; f < 6; ++f) g.face[f] = LBM_WALL;
  apply_geometry(h, &g);
  lbm_params p{};
  p.nu = 1.0 / 6.0;
  p.s_c = 1.0;
  p.s_e = 1.19;
  p.s_q = 1.2;
  p.s_pi = 1.19;
  p.s_t = 0.98;
  apply_params(h, &p);
  g_last_error.clear();
  *out = h;
  return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  DeviceGuard dg(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->d.f) cudaFree(h->d.f);
  if (h->u_prev) cudaFree(h->u_prev);
  if (h->partials) cudaFree(h->partials);
  if (h->stats_host) cudaFreeHost(h->stats_host);
  if (h->staging) cudaFree(h->staging);
  if (h->solid_bytes) cudaFree(h->solid_bytes);
  if (h->solid_links) cudaFree(h->solid_links);
  delete h;
}

int lbm_set_stream(lbm_handle* h, void* cuda_stream) {
  if (int rc = check(h)) return rc;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return LBM_OK;
}

int lbm_set_geometry(lbm_handle* h, const lbm_geom* g) {
  if (int rc = check(h)) return rc;
  if (!g) return fail(LBM_EINVAL, "null geometry");
  return apply_geometry(h, g);
}

int lbm_set_params(lbm_handle* h, const lbm_params* p) {
  if (int rc = check(h)) return rc;
  if (!p) return fail(LBM_EINVAL, "null params");
  return apply_params(h, p);
}

// Device staging space of at least `bytes` (grow-only, kept by the handle).
static int staging(lbm_handle* h, size_t bytes, void** out) {
  if (h->staging_bytes < bytes) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "staging synchronize");
    if (h->staging) cudaFree(h->staging);
    h->bytes -= (int64_t)h->staging_bytes;
    h->staging = nullptr;
    h->staging_bytes = 0;
    e = cudaMalloc(&h->staging, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_ENOMEM, "staging allocation failed");
    }
    h->staging_bytes = bytes;
    h->bytes += (int64_t)bytes;
  }
  *out = h->staging;
  return LBM_OK;
}

// Host arrays are copied into the staging buffer (u first, then p, ...);
// device arrays are used in place.
static int upload(lbm_handle* h, const double* src, size_t count, int on_device,
                  size_t offset, const double** dev) {
  *dev = src;
  if (!src || on_device) return LBM_OK;
  void* base;
  if (int rc = staging(h, (offset + count) * sizeof(double), &base)) return rc;
  double* dst = static_cast<double*>(base) + offset;
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyHostToDevice,
                                  h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
  *dev = dst;
  return LBM_OK;
}

int lbm_set_solid(lbm_handle* h, const uint8_t* solid, int on_device) {
  if (int rc = check(h)) return rc;
  DeviceGuard dg(h->device);
  const size_t N = (size_t)h->d.N;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_solid synchronize");
  if (!solid) {  // back to the plain box
    if (h->solid_bytes) cudaFree(h->solid_bytes);
    if (h->solid_links) cudaFree(h->solid_links);
    if (h->solid_bytes) h->bytes -= (int64_t)(5 * N);
    h->solid_bytes = nullptr;
    h->solid_links = nullptr;
    h->d.solid = nullptr;
    return LBM_OK;
  }
  if (h->d.neq_vel | h->d.neq_pre)
    return fail(LBM_EINVAL, "extrapolation faces do not combine with solid nodes");
  if (!h->solid_bytes) {
    e = cudaMalloc(&h->solid_bytes, N);
    if (e == cudaSuccess) e = cudaMalloc(&h->solid_links, 4 * N);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (h->solid_bytes) cudaFree(h->solid_bytes);
      h->solid_bytes = nullptr;
      h->solid_links = nullptr;
      return fail(LBM_ENOMEM, "solid mask allocation failed");
    }
    h->bytes += (int64_t)(5 * N);
  }
  e = cudaMemcpyAsync(h->solid_bytes, solid, N, on_device ? cudaMemcpyDeviceToDevice
                                                          : cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_solid_links(h->d, h->solid_bytes, h->solid_links, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_solid");
  h->d.solid = h->solid_links;
  return LBM_OK;
}

int lbm_init_equilibrium(lbm_handle* h, const double* u, const double* p, int on_device) {
  if (int rc = check(h)) return rc;
  DeviceGuard dg(h->device);
  const size_t N = (size_t)h->d.N;
  if (!on_device && (u || p)) {  // size the staging buffer once for both
    void* base;
    if (int rc = staging(h, 4 * N * sizeof(double), &base)) return rc;
  }
  const double *du = nullptr, *dp = nullptr;
  int rc = upload(h, u, 3 * N, on_device, 0, &du);
  if (!rc) rc = upload(h, p, N, on_device, 3 * N, &dp);
  if (!rc) {
    cudaError_t e = launch_init(h->d, du, dp, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "init kernel");
  }
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init synchronize");
  h->n = 0;
  h->have_prev = 0;
  h->prev_step = -1;
  h->stats_step = -1;
  h->stats_host[kNumSums - 1] = 0.0;
  return LBM_OK;
}

static int run_reduction(lbm_handle* h) {
  if (!h->u_prev) {
    cudaError_t e = cudaMalloc(&h->u_prev, sizeof(double) * 3 * h->d.N);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_ENOMEM, "snapshot allocation failed");
    }
    h->bytes += (int64_t)sizeof(double) * 3 * h->d.N;
    h->have_prev = 0;
  }
  cudaError_t e = launch_reduce(h->d, h->n, h->u_prev, h->have_prev, h->partials,
                                h->stats_dev, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reduction kernel");
  h->stats_prev_step = h->have_prev ? h->prev_step : -1;
  h->stats_step = h->n;
  h->have_prev = 1;
  h->prev_step = h->n;
  return LBM_OK;
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
  if (int rc = check(h)) return rc;
  if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
  if (static_cast<volatile double*>(h->stats_host)[kNumSums - 1] > 0.0)
    return fail(LBM_EUNSTABLE, "a reduction found non-finite values");
  DeviceGuard dg(h->device);
  const int K = h->params.residual_interval;
  const bool neq = (h->d.neq_vel | h->d.neq_pre) != 0;
  for (int64_t k = 0; k < nsteps; ++k) {
    cudaError_t e = launch_step(h->d, h->n, h->block, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel");
    h->n += 1;
    if (neq) {  // the extrapolation boundaries of the new time level
      e = launch_neq(h->d, h->n, h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "boundary kernel");
    }
    if (K > 0 && h->n % K == 0)
      if (int rc = run_reduction(h)) return rc;
  }
  return LBM_OK;
}

int lbm_get_step(lbm_handle* h, int64_t* n) {
  if (int rc = check(h)) return rc;
  if (!n) return fail(LBM_EINVAL, "null output");
  *n = h->n;
  return LBM_OK;
}

int lbm_set_step(lbm_handle* h, int64_t n) {
  if (int rc = check(h)) return rc;
  if (n < 0) return fail(LBM_EINVAL, "step counter must be >= 0");
  DeviceGuard dg(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_step synchronize");
  h->n = n;
  h->have_prev = 0;
  h->prev_step = -1;
  h->stats_step = -1;
  return LBM_OK;
}

int lbm_read_fields(lbm_handle* h, unsigned mask, void* dst, int dst_on_device, int dtype) {
  if (int rc = check(h)) return rc;
  if (!dst) return fail(LBM_EINVAL, "null destination");
  if (mask == 0 || (mask & ~7u)) return fail(LBM_EINVAL, "bad field mask");
  if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(LBM_EINVAL, "bad dtype");
  DeviceGuard dg(h->device);
  size_t count = 0;
  if (mask & LBM_FIELD_U) count += 3 * (size_t)h->d.N;
  if (mask & LBM_FIELD_P) count += (size_t)h->d.N;
  if (mask & LBM_FIELD_POPULATIONS) count += (size_t)h->d.Q * h->d.N;
  const size_t bytes = count * (dtype == LBM_DTYPE_F64 ? 8 : 4);
  void* target = dst;
  if (!dst_on_device)
    if (int rc = staging(h, bytes, &target)) return rc;
  int rc = LBM_OK;
  cudaError_t e = launch_read(h->d, h->n, mask, target, dtype, h->stream);
  if (e != cudaSuccess) rc = cuda_fail(e, "read kernel");
  if (!rc && !dst_on_device) {
    e = cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync D2H");
  }
  e = cudaStreamSynchronize(h->stream);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "read_fields synchronize");
  return rc;
}

int lbm_write_populations(lbm_handle* h, const double* src, int src_on_device) {
  if (int rc = check(h)) return rc;
  if (!src) return fail(LBM_EINVAL, "null source");
  DeviceGuard dg(h->device);
  const double* dsrc = nullptr;
  int rc = upload(h, src, (size_t)h->d.Q * h->d.N, src_on_device, 0, &dsrc);
  if (!rc) {
    cudaError_t e = launch_write(h->d, h->n, dsrc, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "write kernel");
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "write synchronize");
  if (!rc) {
    h->stats_host[kNumSums - 1] = 0.0;
    h->have_prev = 0;
    h->prev_step = -1;
    h->stats_step = -1;
  }
  return rc;
}

static void fill_stats(lbm_handle* h, lbm_stats* out) {
  const double* s = h->stats_host;
  out->step = h->stats_step;
  out->prev_step = h->stats_prev_step;
  for (int k = 0; k < 3; ++k) {
    out->sum_abs_du[k] = s[k];
    out->sum_abs_u[k] = s[3 + k];
    out->sum_abs_u_prev[k] = s[6 + k];
    out->sum_u[k] = s[10 + k];
  }
  out->sum_P = s[9];
  out->nonfinite = (int64_t)s[kNumSums - 1];
  out->max_abs_u = s[kNumSums];
}

int lbm_reductions(lbm_handle* h, lbm_stats* out) {
  if (int rc = check(h)) return rc;
  if (!out) return fail(LBM_EINVAL, "null output");
  DeviceGuard dg(h->device);
  if (int rc = run_reduction(h)) return rc;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reduction synchronize");
  fill_stats(h, out);
  return LBM_OK;
}

int lbm_read_stats(lbm_handle* h, lbm_stats* out) {
  if (int rc = check(h)) return rc;
  if (!out) return fail(LBM_EINVAL, "null output");
  DeviceGuard dg(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stats synchronize");
  fill_stats(h, out);
  return LBM_OK;
}

int lbm_stats_residual(const lbm_stats* s, int32_t kind, int32_t component, double* r) {
  if (!s || !r) return fail(LBM_EINVAL, "null argument");
  if (kind != LBM_RESIDUAL_CAVITY && (component < 0 || component > 2))
    return fail(LBM_EINVAL, "component must be 0, 1 or 2");
  if (s->prev_step < 0)
    return fail(LBM_EINVAL, "the statistics hold no earlier snapshot (prev_step < 0)");
  double num, den;
  switch (kind) {
    case LBM_RESIDUAL_STEADY:  // Eq. sc: against the earlier time level
      num = s->sum_abs_du[component];
      den = s->sum_abs_u_prev[component];
      break;
    case LBM_RESIDUAL_PERIODIC:  // Eq. cr: against the later time level
      num = s->sum_abs_du[component];
      den = s->sum_abs_u[component];
      break;
    case LBM_RESIDUAL_CAVITY:  // Eq. cavity_creterion: every component, later level
      num = s->sum_abs_du[0] + s->sum_abs_du[1] + s->sum_abs_du[2];
      den = s->sum_abs_u[0] + s->sum_abs_u[1] + s->sum_abs_u[2];
      break;
    default: return fail(LBM_EINVAL, "unknown residual kind");
  }
  *r = den > 0.0 ? num / den : (num == 0.0 ? 0.0 : HUGE_VAL);
  return LBM_OK;
}

int lbm_residual(lbm_handle* h, int32_t kind, int32_t component, double* r) {
  if (int rc = check(h)) return rc;
  if (!r) return fail(LBM_EINVAL, "null output");
  DeviceGuard dg(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "residual synchronize");
  if (h->stats_step < 0) return fail(LBM_EINVAL, "no reduction has run yet");
  lbm_stats s;
  fill_stats(h, &s);
  return lbm_stats_residual(&s, kind, component, r);
}

int lbm_set_launch(lbm_handle* h, const lbm_launch* l) {
  if (int rc = check(h)) return rc;
  if (!l) return fail(LBM_EINVAL, "null launch");
  if (l->bx < 32 || l->bx % 32 != 0 || l->by < 1 || (int64_t)l->bx * l->by > 256)
    return fail(LBM_EINVAL, "block must be bx (multiple of 32) x by with bx*by <= 256");
  if (l->cells_per_thread != 1 && l->cells_per_thread != 2)
    return fail(LBM_EINVAL, "cells_per_thread must be 1 or 2");
  if (l->cells_per_thread == 2 && h->d.storage == LBM_STORAGE_F64)
    return fail(LBM_EINVAL, "two cells per thread needs FP32 arithmetic (not FP64 storage)");
  h->block = {l->bx, l->by, l->cells_per_thread, h->block.pdl};
  return LBM_OK;
}

int lbm_set_overlap(lbm_handle* h, int32_t enable) {
  if (int rc = check(h)) return rc;
  h->block.pdl = enable ? 1 : 0;
  return LBM_OK;
}

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::pair<BlockShape, double>> g_tune_cache;

const BlockShape kCandidates[] = {{32, 1, 1},  {32, 2, 1}, {32, 4, 1}, {32, 8, 1},
                                  {64, 1, 1},  {64, 2, 1}, {64, 4, 1}, {128, 1, 1},
                                  {128, 2, 1}, {256, 1, 1}, {32, 2, 2}, {64, 1, 2},
                                  {64, 2, 2},  {128, 1, 2}};
}  // namespace

int lbm_autotune(lbm_handle* h, int32_t trials, lbm_launch* chosen, double* ms) {
  if (int rc = check(h)) return rc;
  DeviceGuard dg(h->device);
  const auto key =
      std::make_tuple(h->d.Q, h->d.storage, h->d.rounding, h->d.nx, h->d.ny, h->d.nz);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && trials <= 0) {
      const BlockShape& c = it->second.first;
      h->block = {c.bx, c.by, c.cpt, h->block.pdl};
      if (chosen) *chosen = {h->block.bx, h->block.by, h->block.cpt};
      if (ms) *ms = it->second.second;
      return LBM_OK;
    }
  }
  if (trials <= 0) trials = 8;
  trials += trials & 1;  // even: equal numbers of even and odd steps
  const size_t fbytes = (size_t)h->d.N * h->d.Q * storage_bytes(h->d.storage);
  void* saved = nullptr;
  cudaError_t e = cudaMalloc(&saved, fbytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_ENOMEM, "autotune: no memory for the saved state");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LBM_OK;
  e = cudaMemcpyAsync(saved, h->d.f, fbytes, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  BlockShape best = h->block;
  double best_ms = 1e300;
  const int64_t n0 = h->n;
  const int xmax = ((h->d.nx + 31) / 32) * 32;
  for (BlockShape b : kCandidates) {
    if (e != cudaSuccess) break;
    b.pdl = h->block.pdl;
    if (b.bx * b.cpt > xmax && b.bx > 32) continue;
    if (b.cpt == 2 && (h->d.storage == LBM_STORAGE_F64 || h->d.Q == 26 ||
                       (int64_t)h->d.Q * h->d.N >= (int64_t(1) << 31)))
      continue;
    int64_t n = n0;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = launch_step(h->d, n++, b, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int k = 0; k < trials && e == cudaSuccess; ++k) e = launch_step(h->d, n++, b, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && t / trials < best_ms) {
      best_ms = t / trials;
      best = b;
    }
    // back to the saved state (and parity) before the next candidate
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->d.f, saved, fbytes, cudaMemcpyDeviceToDevice, h->stream);
  }
  if (e != cudaSuccess) rc = cuda_fail(e, "autotune");
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  if (!rc && e2 != cudaSuccess) rc = cuda_fail(e2, "autotune synchronize");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(saved);
  h->n = n0;
  if (rc) return rc;
  h->block = best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {best, best_ms};
  }
  if (chosen) *chosen = {best.bx, best.by, best.cpt};
  if (ms) *ms = best_ms;
  return LBM_OK;
}

int lbm_get_launch(lbm_handle* h, lbm_launch* out) {
  if (int rc = check(h)) return rc;
  if (!out) return fail(LBM_EINVAL, "null output");
  *out = {h->block.bx, h->block.by, h->block.cpt};
  return LBM_OK;
}

int lbm_device_populations(lbm_handle* h, void** ptr, int64_t* bytes) {
  if (int rc = check(h)) return rc;
  if (!ptr || !bytes) return fail(LBM_EINVAL, "null output");
  *ptr = h->d.f;
  *bytes = h->d.N * h->d.Q * (int64_t)storage_bytes(h->d.storage);
  return LBM_OK;
}

int lbm_memory_bytes(lbm_handle* h, int64_t* bytes) {
  if (int rc = check(h)) return rc;
  if (!bytes) return fail(LBM_EINVAL, "null output");
  *bytes = h->bytes;
  return LBM_OK;
}

}  // extern "C"
