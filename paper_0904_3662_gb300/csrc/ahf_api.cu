// Host side of libahfgpu: the C ABI, argument validation, the size-class
// scheduler and the context's device workspace.
//
// Scheduling.  Haloes are independent units (the paper's parallel version
// relies on the same fact: no communication during the analysis, Sect. 2.2).
// Each halo goes to a size class by its candidate count: three on-chip
// variants (one CTA per halo, everything in shared memory) and, above the
// largest on-chip capacity, the multi-CTA class that streams its particles
// through HBM.  Within a class the haloes are processed largest first by
// persistent CTAs pulling from a device counter (longest-processing-time
// order), so the biggest halo starts first and the tail is short.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "ahf_internal.h"

using namespace ahf;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define AHF_CUDA(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(AHF_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                         \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// A bump allocator over the context's device workspace, rebuilt per call.
struct Bump {
  char* base = nullptr;
  size_t used = 0;
  size_t cap = 0;
  template <typename T>
  T* take(size_t count) {
    used = align_up(used, 256);
    T* p = reinterpret_cast<T*>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

}  // namespace

struct ahf_ctx {
  int device = 0;
  int sms = 0;
  char* ws = nullptr;            // device workspace
  size_t ws_bytes = 0;
  int* err_dev = nullptr;        // device error word
  int* err_host = nullptr;       // pinned mirror
  cudaEvent_t last = nullptr;    // end of the previous call's device work
  bool last_valid = false;
  int64_t onchip_max = 8192;
  int64_t wait_limit = 1 << 22;
  std::mutex mu;
  // pinned staging for host descriptors
  void* pin = nullptr;
  size_t pin_bytes = 0;
};

namespace {

int ensure_pinned(ahf_ctx* c, size_t bytes) {
  if (bytes <= c->pin_bytes) return AHF_OK;
  if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
  if (c->pin) cudaFreeHost(c->pin);
  c->pin = nullptr;
  c->pin_bytes = 0;
  size_t want = std::max(bytes, (size_t)1 << 20);
  if (cudaMallocHost(&c->pin, want) != cudaSuccess) return fail(AHF_ERR_NOMEM, "pinned staging of %zu bytes", want);
  c->pin_bytes = want;
  return AHF_OK;
}

int ensure_workspace(ahf_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return AHF_OK;
  if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
  if (c->ws) cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_bytes = 0;
  size_t want = std::max(align_up(bytes + bytes / 8, 1 << 20), (size_t)1 << 22);
  if (cudaMalloc(&c->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(AHF_ERR_NOMEM, "device workspace of %zu bytes", want);
  }
  c->ws_bytes = want;
  return AHF_OK;
}

int ceil_log2(double x) {
  int e = 0;
  while (e < 1100 && std::ldexp(1.0, e) <= x) ++e;
  return e;
}

struct Plan {
  std::vector<HaloDev> hd;     // reordered: class 0, 1, 2 (on-chip), then grid class
  int n_class[4] = {0, 0, 0, 0};
  long long grid_flat = 0;
  FrameDev frame;
};

int validate(const ahf_particles* p, const ahf_halo* halos, int64_t n_halos, const ahf_params* prm,
             const ahf_result* out, const int64_t* bound_idx) {
  if (!p || !prm) return fail(AHF_ERR_INVALID, "particles and params must not be NULL");
  if (n_halos < 0) return fail(AHF_ERR_INVALID, "n_halos < 0");
  if (n_halos > 0 && (!halos || !out || !bound_idx))
    return fail(AHF_ERR_INVALID, "halos, out and bound_idx must not be NULL");
  if (n_halos > (int64_t)0x7fffffff) return fail(AHF_ERR_INVALID, "n_halos above 2^31-1");
  if (p->n < 0) return fail(AHF_ERR_INVALID, "particle count < 0");
  if (p->n > 0 && (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz))
    return fail(AHF_ERR_INVALID, "coordinate or velocity array is NULL");
  if (p->coord_type != AHF_COORD_F64 && p->coord_type != AHF_COORD_F32_REL && p->coord_type != AHF_COORD_F32_BOX)
    return fail(AHF_ERR_INVALID, "unknown coord_type %d", p->coord_type);
  if (p->reserved != 0) return fail(AHF_ERR_INVALID, "reserved field must be 0");
  if (!p->m && !(p->m0 >= 0.0 && std::isfinite(p->m0))) return fail(AHF_ERR_INVALID, "m0 must be finite and >= 0");
  if (prm->max_iter < 1) return fail(AHF_ERR_INVALID, "max_iter must be >= 1");
  if (prm->precision != AHF_PREC_MIXED) return fail(AHF_ERR_INVALID, "precision mode %d not available", prm->precision);
  if (!(prm->G > 0.0) || !std::isfinite(prm->G)) return fail(AHF_ERR_INVALID, "G must be > 0");
  if (!std::isfinite(prm->H)) return fail(AHF_ERR_INVALID, "H must be finite");
  if (!(prm->delta_rho > 0.0) || !std::isfinite(prm->delta_rho)) return fail(AHF_ERR_INVALID, "delta_rho must be > 0");
  if (!(prm->r_soft >= 0.0) || !std::isfinite(prm->r_soft)) return fail(AHF_ERR_INVALID, "r_soft must be >= 0");
  if (!(prm->box >= 0.0) || !std::isfinite(prm->box)) return fail(AHF_ERR_INVALID, "box must be >= 0");
  if (!(prm->band >= 0.0) || !(prm->band < 1.0)) return fail(AHF_ERR_INVALID, "band must be in [0, 1)");
  return AHF_OK;
}

// Check slots: in range of the slot space and not shared between haloes.
int validate_slots(const ahf_halo* halos, int64_t n_halos, int64_t n_slots, bool have_members) {
  std::vector<std::pair<int64_t, int64_t>> iv;
  iv.reserve((size_t)n_halos);
  for (int64_t h = 0; h < n_halos; ++h) {
    const ahf_halo& H = halos[h];
    if (H.count < 0 || H.offset < 0) return fail(AHF_ERR_INVALID, "halo %lld: negative offset or count", (long long)h);
    if (H.count > (int64_t)0x7fffffff) return fail(AHF_ERR_INVALID, "halo %lld: count above 2^31-1", (long long)h);
    if (!have_members && H.offset + H.count > n_slots)
      return fail(AHF_ERR_INVALID, "halo %lld: slots [%lld, %lld) beyond %lld particles", (long long)h,
                  (long long)H.offset, (long long)(H.offset + H.count), (long long)n_slots);
    if (!(std::isfinite(H.cx) && std::isfinite(H.cy) && std::isfinite(H.cz)))
      return fail(AHF_ERR_INVALID, "halo %lld: centre not finite", (long long)h);
    if (std::isnan(H.radius)) return fail(AHF_ERR_INVALID, "halo %lld: radius is NaN", (long long)h);
    if (H.count > 0) iv.emplace_back(H.offset, H.offset + H.count);
  }
  std::sort(iv.begin(), iv.end());
  for (size_t i = 1; i < iv.size(); ++i)
    if (iv[i].first < iv[i - 1].second) return fail(AHF_ERR_INVALID, "haloes share candidate slots");
  return AHF_OK;
}

int make_plan(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos, const ahf_params* prm,
              Plan& P) {
  // fixed-point frame: every member coordinate and centre stays below 2^(61-frac)
  double maxabs = prm->box;
  for (int64_t h = 0; h < n_halos; ++h) {
    const ahf_halo& H = halos[h];
    const double cm = std::max(std::fabs(H.cx), std::max(std::fabs(H.cy), std::fabs(H.cz)));
    const double rad = std::isfinite(H.radius) ? std::fabs(H.radius) : 0.0;
    maxabs = std::max(maxabs, cm + rad);
  }
  if (p->coord_type == AHF_COORD_F32_REL) maxabs = std::max(maxabs, 1.0);
  int frac = 60 - ceil_log2(maxabs + 1.0);
  if (frac > 200) frac = 200;
  if (frac < -200) frac = -200;
  P.frame.frac = frac;
  P.frame.box = prm->box;
  P.frame.boxfix = prm->box > 0.0 ? (long long)std::llround(std::ldexp(prm->box, frac)) : 0;

  const int cap0 = onchip_capacity(0), cap1 = onchip_capacity(1);
  const int cap2 = (int)std::min<int64_t>(c->onchip_max, onchip_capacity(2));
  std::vector<int> cls((size_t)n_halos);
  for (int64_t h = 0; h < n_halos; ++h) {
    const int64_t n = halos[h].count;
    cls[h] = n <= std::min<int64_t>(cap0, c->onchip_max) ? 0
             : n <= std::min<int64_t>(cap1, c->onchip_max) ? 1
             : n <= cap2 ? 2 : 3;
    P.n_class[cls[h]]++;
  }
  std::vector<int> order((size_t)n_halos);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (cls[a] != cls[b]) return cls[a] < cls[b];
    return halos[a].count > halos[b].count;
  });
  P.hd.resize((size_t)n_halos);
  long long gbase = 0;
  for (int64_t k = 0; k < n_halos; ++k) {
    const int h = order[k];
    const ahf_halo& H = halos[h];
    HaloDev& d = P.hd[k];
    d.c[0] = H.cx; d.c[1] = H.cy; d.c[2] = H.cz;
    for (int a = 0; a < 3; ++a) d.cfix[a] = (long long)std::llround(std::ldexp(d.c[a], frac));
    const double R = H.radius;
    d.R2 = std::isinf(R) ? INFINITY : R * R;
    d.R2lo = (float)(d.R2 * (1.0 - 4e-6));
    d.R2hi = (float)(d.R2 * (1.0 + 4e-6));
    if (std::isinf(d.R2)) { d.R2lo = INFINITY; d.R2hi = INFINITY; }
    d.offset = H.offset;
    d.count = H.count;
    d.index = h;
    d.pad = 0;
    d.gbase = 0;
    if (cls[h] == 3) { d.gbase = gbase; gbase += H.count; }
  }
  P.grid_flat = gbase;
  return AHF_OK;
}

ParamsDev to_dev(const ahf_params* prm) {
  ParamsDev d;
  d.G = prm->G; d.H = prm->H; d.delta_rho = prm->delta_rho; d.r_soft = prm->r_soft; d.band = prm->band;
  d.Gf = (float)prm->G; d.Hf = (float)prm->H; d.r_soft_f = (float)prm->r_soft; d.band_f = (float)prm->band;
  d.crit = prm->delta_rho * (4.0 * M_PI / 3.0);
  d.crit_f = (float)d.crit;
  d.max_iter = prm->max_iter;
  d.precision = prm->precision;
  return d;
}

ParticlesDev to_dev(const ahf_particles* p) {
  ParticlesDev d;
  d.x = p->x; d.y = p->y; d.z = p->z; d.vx = p->vx; d.vy = p->vy; d.vz = p->vz; d.m = p->m;
  d.m0 = p->m0; d.m0f = (float)p->m0; d.coord_type = p->coord_type; d.n = p->n;
  return d;
}

int begin_call(ahf_ctx* c, cudaStream_t s) {
  AHF_CUDA(cudaSetDevice(c->device));
  if (c->last_valid) AHF_CUDA(cudaStreamWaitEvent(s, c->last, 0));
  return AHF_OK;
}

int end_call(ahf_ctx* c, cudaStream_t s) {
  AHF_CUDA(cudaEventRecord(c->last, s));
  c->last_valid = true;
  return AHF_OK;
}

int unbind_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx, void* phi,
                int32_t* removed_iter, cudaStream_t s) {
  int rc = validate(p, halos, n_halos, prm, out, bound_idx);
  if (rc) return rc;
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  if ((rc = validate_slots(halos, n_halos, n_slots, member_idx != nullptr))) return rc;
  if (n_halos == 0) return AHF_OK;
  Plan P;
  if ((rc = make_plan(c, p, halos, n_halos, prm, P))) return rc;
  if (P.n_class[3] > 0)
    return fail(AHF_ERR_INVALID, "haloes above %lld candidates need the multi-CTA class", (long long)c->onchip_max);

  // workspace
  size_t need = align_up(sizeof(HaloDev) * (size_t)n_halos, 256) + 4096;
  if ((rc = ensure_workspace(c, need))) return rc;
  if ((rc = ensure_pinned(c, sizeof(HaloDev) * (size_t)n_halos + 256))) return rc;
  if ((rc = begin_call(c, s))) return rc;
  Bump B{c->ws, 0, c->ws_bytes};
  HaloDev* hd = B.take<HaloDev>((size_t)n_halos);
  int* queues = B.take<int>(16);
  // the pinned staging buffer is reused by later calls: wait for its last copy
  if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
  std::memcpy(c->pin, P.hd.data(), sizeof(HaloDev) * (size_t)n_halos);
  AHF_CUDA(cudaMemcpyAsync(hd, c->pin, sizeof(HaloDev) * (size_t)n_halos, cudaMemcpyHostToDevice, s));
  AHF_CUDA(cudaMemsetAsync(queues, 0, 16 * sizeof(int), s));

  OutputsDev O;
  O.res = out; O.bound_idx = (long long*)bound_idx; O.phi = phi; O.removed_iter = removed_iter;
  O.member_idx = (const long long*)member_idx; O.n_slots = n_slots; O.err = c->err_dev;
  const ParticlesDev pd = to_dev(p);
  const ParamsDev prd = to_dev(prm);
  int first = 0;
  for (int v = 0; v < 3; ++v) {
    const int n = P.n_class[v];
    if (n > 0) {
      OnchipLaunch L;
      L.p = pd; L.frame = P.frame; L.prm = prd; L.out = O;
      L.halos = hd + first; L.n_halos = n; L.queue = queues + v;
      const int grid = std::min(n, onchip_max_grid(v, c->device));
      AHF_CUDA(launch_onchip(L, v, grid, s));
    }
    first += n;
  }
  return end_call(c, s);
}

}  // namespace

extern "C" {

int ahf_version(void) { return 100; }

const char* ahf_last_error(void) { return g_last_error.c_str(); }

int ahf_create(ahf_ctx** ctx, int device) {
  if (!ctx) return fail(AHF_ERR_INVALID, "ctx is NULL");
  *ctx = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return fail(AHF_ERR_INVALID, "no CUDA device %d", device);
  }
  ahf_ctx* c = new (std::nothrow) ahf_ctx();
  if (!c) return fail(AHF_ERR_NOMEM, "context allocation");
  c->device = device;
  int rc = AHF_OK;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = fail(AHF_ERR_CUDA, "cudaSetDevice(%d)", device); break; }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->err_dev, sizeof(int)) != cudaSuccess) { rc = fail(AHF_ERR_NOMEM, "error word"); break; }
    if (cudaMemset(c->err_dev, 0, sizeof(int)) != cudaSuccess) { rc = fail(AHF_ERR_CUDA, "memset"); break; }
    if (cudaMallocHost(&c->err_host, sizeof(int)) != cudaSuccess) { rc = fail(AHF_ERR_NOMEM, "pinned word"); break; }
    if (cudaEventCreateWithFlags(&c->last, cudaEventDisableTiming) != cudaSuccess) {
      rc = fail(AHF_ERR_CUDA, "event");
      break;
    }
  } while (0);
  if (rc != AHF_OK) {
    cudaGetLastError();
    ahf_destroy(c);
    return rc;
  }
  *ctx = c;
  return AHF_OK;
}

int ahf_destroy(ahf_ctx* c) {
  if (!c) return AHF_OK;
  cudaSetDevice(c->device);
  if (c->last_valid) cudaEventSynchronize(c->last);
  if (c->ws) cudaFree(c->ws);
  if (c->err_dev) cudaFree(c->err_dev);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->pin) cudaFreeHost(c->pin);
  if (c->last) cudaEventDestroy(c->last);
  delete c;
  return AHF_OK;
}

int ahf_set_option(ahf_ctx* c, int option, int64_t value) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  switch (option) {
    case AHF_OPT_ONCHIP_MAX:
      if (value < 0 || value > onchip_capacity(2)) return fail(AHF_ERR_INVALID, "onchip max out of range");
      c->onchip_max = value;
      return AHF_OK;
    case AHF_OPT_WAIT_LIMIT:
      if (value < 0) return fail(AHF_ERR_INVALID, "wait limit < 0");
      c->wait_limit = value;
      return AHF_OK;
    default:
      return fail(AHF_ERR_INVALID, "unknown option %d", option);
  }
}

int ahf_get_option(ahf_ctx* c, int option, int64_t* value) {
  if (!c || !value) return fail(AHF_ERR_INVALID, "NULL argument");
  switch (option) {
    case AHF_OPT_ONCHIP_MAX: *value = c->onchip_max; return AHF_OK;
    case AHF_OPT_WAIT_LIMIT: *value = c->wait_limit; return AHF_OK;
    default: return fail(AHF_ERR_INVALID, "unknown option %d", option);
  }
}

int ahf_sync(ahf_ctx* c) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  AHF_CUDA(cudaSetDevice(c->device));
  if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
  AHF_CUDA(cudaMemcpy(c->err_host, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  const int e = *c->err_host;
  if (e) AHF_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
  if (e & ERR_TIMEOUT) return fail(AHF_ERR_TIMEOUT, "a bounded device wait gave up");
  if (e & ERR_BAD_INDEX) return fail(AHF_ERR_INVALID, "a member index was out of range");
  if (e & ERR_CAPACITY) return fail(AHF_ERR_INVALID, "a halo exceeded its size class");
  return AHF_OK;
}

int ahf_unbind_batch(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                     const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx,
                     void* phi, int32_t* removed_iter, void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return unbind_impl(c, p, halos, n_halos, member_idx, prm, out, bound_idx, phi, removed_iter,
                     (cudaStream_t)stream);
}

}  // extern "C"
