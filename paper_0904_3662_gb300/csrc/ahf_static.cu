// ahf_unbind_batch_static: the on-chip unbinding class without any memory
// allocation.
//
// Some callers cannot let a library allocate: applications that have handed
// the whole GPU memory to their own allocator (a framework's caching
// allocator, a serving engine's pre-partitioned pool), and latency-critical
// loops that must never block in cudaMalloc / cudaFree, which synchronise
// the device.  This entry point uses no context: its scratch (the halo
// descriptors and work counters the on-chip kernel reads) lives in one
// fixed-size array in device global memory, declared below, and its host
// side stages descriptors through a fixed-size host array.  It calls no
// cudaMalloc, cudaMallocHost, cudaFree or any other allocating routine.
//
// Limits: at most AHF_STATIC_MAX_HALOS haloes per call and at most
// AHF_STATIC_MAX_COUNT candidate slots per halo (the on-chip capacity).
// Every call on a device shares the one scratch array, which keeps the last
// call's contents; each call clears the counters it needs.  Two calls whose
// device work overlaps (different streams, no ordering between them) race
// on the array and their results are undefined.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "ahf_internal.h"

namespace ahf {
namespace {

constexpr size_t STATIC_COUNTER_BYTES = 256;   // 3 queue counters + the error word
constexpr size_t STATIC_SCRATCH_BYTES =
    STATIC_COUNTER_BYTES + sizeof(HaloDev) * (size_t)AHF_STATIC_MAX_HALOS;

// The scratch array (about 3.8 MiB, held by every GPU that loads the
// library until the process exits).  In host code this name is only a
// host-side stand-in; kernels receive the device address looked up below.
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;                               // guards the tables and the host staging
void* g_scratch_addr[MAX_DEVICES] = {};        // device address of the array, per device
int g_grid[MAX_DEVICES][3] = {};               // resident CTAs of the three variants, per device

// Host staging (fixed size, no allocation): descriptors in launch order.
HaloDev g_stage[AHF_STATIC_MAX_HALOS];
int g_order[AHF_STATIC_MAX_HALOS];

int fail_static(int code, const char* msg) {
  set_last_error_static(msg);     // a string literal: nothing is allocated
  return code;
}

// The device error word of this call (bad member indices) into the caller's
// int, cleared for the next call.
__global__ void report_error_word(int* word, int32_t* out) {
  const int e = *word;
  *out = e ? AHF_ERR_INVALID : AHF_OK;
  *word = 0;
}


}  // namespace

}  // namespace ahf

using namespace ahf;

extern "C" int ahf_unbind_batch_static(const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                                       const int64_t* member_idx, const ahf_params* prm, ahf_result* out,
                                       int64_t* bound_idx, void* phi, int32_t* removed_iter, int32_t* error_out,
                                       void* stream) {
  // ---- arguments (no CUDA call before they are known to be valid) ----
  if (!p || !prm) return fail_static(AHF_ERR_INVALID, "particles and params must not be NULL");
  if (n_halos < 0) return fail_static(AHF_ERR_INVALID, "n_halos < 0");
  if (n_halos > AHF_STATIC_MAX_HALOS)
    return fail_static(AHF_ERR_INVALID, "ahf_unbind_batch_static takes at most AHF_STATIC_MAX_HALOS haloes");
  if (n_halos > 0 && (!halos || !out || !bound_idx))
    return fail_static(AHF_ERR_INVALID, "halos, out and bound_idx must not be NULL");
  if (p->n < 0 || (p->n > 0 && (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz)))
    return fail_static(AHF_ERR_INVALID, "bad particle store");
  if (p->coord_type != AHF_COORD_F64 && p->coord_type != AHF_COORD_F32_REL && p->coord_type != AHF_COORD_F32_BOX)
    return fail_static(AHF_ERR_INVALID, "unknown coord_type");
  if (p->reserved != 0) return fail_static(AHF_ERR_INVALID, "reserved field must be 0");
  if (!p->m && !(p->m0 >= 0.0 && std::isfinite(p->m0))) return fail_static(AHF_ERR_INVALID, "m0 must be >= 0");
  if (prm->max_iter < 1) return fail_static(AHF_ERR_INVALID, "max_iter must be >= 1");
  if (prm->precision != AHF_PREC_MIXED) return fail_static(AHF_ERR_INVALID, "only AHF_PREC_MIXED");
  if (p->u_th) return fail_static(AHF_ERR_INVALID, "no gas thermal energies (u_th) here");
  if (prm->variant & ~(AHF_VAR_VBULK_INITIAL | AHF_VAR_RISE_EDGE))
    return fail_static(AHF_ERR_INVALID, "only the AHF_VAR_VBULK_INITIAL and AHF_VAR_RISE_EDGE variants");
  if (prm->reserved != 0) return fail_static(AHF_ERR_INVALID, "params.reserved must be 0");
  if (!(prm->G > 0.0) || !std::isfinite(prm->G) || !std::isfinite(prm->H) || !(prm->delta_rho > 0.0) ||
      !std::isfinite(prm->delta_rho) || !(prm->r_soft >= 0.0) || !std::isfinite(prm->r_soft) ||
      !(prm->box >= 0.0) || !std::isfinite(prm->box) || !(prm->band >= 0.0) || !(prm->band < 1.0))
    return fail_static(AHF_ERR_INVALID, "bad parameter value");
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  for (int64_t h = 0; h < n_halos; ++h) {
    const ahf_halo& H = halos[h];
    if (H.count < 0 || H.offset < 0) return fail_static(AHF_ERR_INVALID, "negative offset or count");
    if (H.count > AHF_STATIC_MAX_COUNT)
      return fail_static(AHF_ERR_INVALID, "a halo has more than AHF_STATIC_MAX_COUNT candidates");
    if (!member_idx && H.offset + H.count > n_slots) return fail_static(AHF_ERR_INVALID, "slots beyond the store");
    if (!(std::isfinite(H.cx) && std::isfinite(H.cy) && std::isfinite(H.cz) && std::isfinite(H.radius)))
      return fail_static(AHF_ERR_INVALID, "centre and radius must be finite");
  }
  if (n_halos == 0) return AHF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // the descriptor copy below reads g_stage, which every later call
  // overwrites: a captured copy would replay with another call's haloes
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return fail_static(AHF_ERR_CUDA, "cudaStreamIsCapturing failed");
  }
  if (cap != cudaStreamCaptureStatusNone)
    return fail_static(AHF_ERR_INVALID, "ahf_unbind_batch_static does not run while its stream is being captured");

  std::lock_guard<std::mutex> guard(g_mu);
  // slots must not be shared: order by offset in the fixed index array
  for (int64_t h = 0; h < n_halos; ++h) g_order[h] = (int)h;
  std::sort(g_order, g_order + n_halos, [&](int a, int b) { return halos[a].offset < halos[b].offset; });
  int64_t end = -1;
  for (int64_t k = 0; k < n_halos; ++k) {
    const ahf_halo& H = halos[g_order[k]];
    if (H.count == 0) continue;
    if (H.offset < end) return fail_static(AHF_ERR_INVALID, "haloes share candidate slots");
    end = H.offset + H.count;
  }

  // ---- scratch address of this device (looked up once per device) ----
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return fail_static(AHF_ERR_CUDA, "cudaGetDevice failed");
  }
  if (!g_scratch_addr[dev]) {
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_static_scratch) != cudaSuccess || !a) {
      cudaGetLastError();
      return fail_static(AHF_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    g_scratch_addr[dev] = a;
    for (int v = 0; v < 3; ++v) g_grid[dev][v] = onchip_max_grid(v, dev);
  }
  for (int v = 0; v < 3; ++v)
    if (g_grid[dev][v] <= 0) return fail_static(AHF_ERR_CUDA, "an on-chip variant cannot run on this device");
  char* scratch = (char*)g_scratch_addr[dev];
  int* counters = (int*)scratch;                                 // [0..2] queues, [8] error word
  HaloDev* hd = (HaloDev*)(scratch + STATIC_COUNTER_BYTES);

  // ---- descriptors: on-chip variants by size, largest first ----
  const int caps[3] = {onchip_capacity(0), onchip_capacity(1), onchip_capacity(2)};
  auto cls = [&](int64_t c) { return c <= caps[0] ? 0 : (c <= caps[1] ? 1 : 2); };
  std::sort(g_order, g_order + n_halos, [&](int a, int b) {
    const int ca = cls(halos[a].count), cb = cls(halos[b].count);
    if (ca != cb) return ca < cb;
    if (halos[a].count != halos[b].count) return halos[a].count > halos[b].count;
    return a < b;
  });
  int n_class[3] = {0, 0, 0};
  for (int64_t k = 0; k < n_halos; ++k) {
    const int h = g_order[k];
    const ahf_halo& H = halos[h];
    n_class[cls(H.count)]++;
    fill_halo_dev(H, p->coord_type, prm->box, h, g_stage[k]);
  }
  // pageable source: the copy has taken the bytes when the call returns
  if (cudaMemcpyAsync(hd, g_stage, sizeof(HaloDev) * (size_t)n_halos, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(counters, 0, STATIC_COUNTER_BYTES, s) != cudaSuccess) {
    cudaGetLastError();
    return fail_static(AHF_ERR_CUDA, "staging the descriptors failed");
  }

  OnchipLaunch L;
  L.p.x = p->x; L.p.y = p->y; L.p.z = p->z; L.p.vx = p->vx; L.p.vy = p->vy; L.p.vz = p->vz; L.p.m = p->m;
  L.p.m0 = p->m0; L.p.m0f = (float)p->m0; L.p.coord_type = p->coord_type; L.p.n = p->n;
  L.frame.box = prm->box;
  L.prm.G = prm->G; L.prm.H = prm->H; L.prm.delta_rho = prm->delta_rho; L.prm.r_soft = prm->r_soft;
  L.prm.band = prm->band;
  L.prm.Gf = (float)prm->G; L.prm.Hf = (float)prm->H; L.prm.r_soft_f = (float)prm->r_soft;
  L.prm.band_f = (float)prm->band;
  L.prm.crit = prm->delta_rho * (4.0 * M_PI / 3.0);
  L.prm.crit_f = (float)L.prm.crit;
  L.prm.inv_crit = 1.0 / L.prm.crit;
  L.prm.max_iter = prm->max_iter;
  L.prm.precision = prm->precision;
  L.prm.vbulk_initial = (prm->variant & AHF_VAR_VBULK_INITIAL) ? 1 : 0;
  L.prm.rise_edge = (prm->variant & AHF_VAR_RISE_EDGE) ? 1 : 0;
  L.out.res = out; L.out.bound_idx = (long long*)bound_idx; L.out.phi = phi; L.out.removed_iter = removed_iter;
  L.out.member_idx = (const long long*)member_idx; L.out.n_slots = n_slots; L.out.err = counters + 8;
  L.rows.prof = nullptr; L.rows.factor = nullptr; L.rows.factor_f = nullptr; L.rows.n_bins = 0;
  L.trace = nullptr;
  L.variant = 0;
  L.rec = nullptr;                  // no scratch for records: the fill re-reads the particle store
  // variants in the order the descriptors were staged; each class is its own queue
  int base = 0;
  for (int v = 0; v < 3; ++v) {
    const int n = n_class[v];
    if (n > 0) {
      L.halos = hd + base;
      L.n_halos = n;
      L.queue = counters + v;
      const int grid = std::min(n, g_grid[dev][v]);
      if (launch_onchip(L, v, grid, s) != cudaSuccess) {
        cudaGetLastError();
        return fail_static(AHF_ERR_CUDA, "kernel launch failed");
      }
    }
    base += n;
  }
  if (error_out) {
    report_error_word<<<1, 1, 0, s>>>(L.out.err, error_out);
    if (cudaGetLastError() != cudaSuccess) return fail_static(AHF_ERR_CUDA, "kernel launch failed");
  }
  return AHF_OK;
}
