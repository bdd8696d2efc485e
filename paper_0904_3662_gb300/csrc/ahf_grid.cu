// Multi-CTA class: haloes too large for one CTA's shared memory.
//
// The haloes of this class share flat arrays (halo k owns [gbase_k,
// gbase_k + count_k)) cut into tiles of GRID_TILE elements that never cross
// a halo.  The steps are those of the on-chip class (Sect. 2.1, Appendix A),
// each a grid-wide kernel:
//   prepare   recentre, sphere test, radius key, exponent maxima
//   sort      segmented stable LSD radix sort (per pass: tile histograms,
//             per-(halo, digit) scans over tiles, per-halo digit bases,
//             stable tile scatter)
//   fill      sorted SoA (w.x, w.y, w.z, m) + radius, exact sum m v
//   iterate   tile sums -> per-halo tile scan -> phi / escape test / removal
//             -> per-halo bookkeeping, repeated while any halo changes
//   finish    final scan, bound list and phi, virial crossing, records
// Every cross-tile combination goes through a separate kernel, so no CTA
// ever waits on another one.
#include <cstdint>

#include "ahf_device.cuh"

namespace ahf {
namespace {

constexpr int T = GRID_THREADS;         // 256
constexpr int TILE = GRID_TILE;         // 2048
constexpr int IPT = TILE / T;           // 8 elements per thread
constexpr int NWARP = T / 32;

// Precision of the per-particle arithmetic.  float: the mixed mode (FP32
// radius key, FP32 phi and escape test).  double: the all-FP64 mode (FP64
// offsets, radius key, phi and escape test); sums stay exact fixed point.
struct alignas(32) D4 {
  double x, y, z, w;
};
template <typename R>
struct Prec;
template <>
struct Prec<float> {
  using Key = uint32_t;
  using V4 = float4;
  static constexpr int KEY_BYTES = 4;
};
template <>
struct Prec<double> {
  using Key = unsigned long long;
  using V4 = D4;
  static constexpr int KEY_BYTES = 8;
};

__device__ __forceinline__ uint32_t key_of(float r) { return __float_as_uint(r); }
__device__ __forceinline__ unsigned long long key_of(double r) { return (unsigned long long)__double_as_longlong(r); }
__device__ __forceinline__ float real_of(uint32_t k, float) { return __uint_as_float(k); }
__device__ __forceinline__ double real_of(unsigned long long k, double) { return __longlong_as_double((long long)k); }
__device__ __forceinline__ long long fix_real(float x, int s) { return fix_from_float(x, s); }
__device__ __forceinline__ long long fix_real(double x, int s) { return fix_from_double(x, s); }
__device__ __forceinline__ int exp_of_bits(unsigned long long b, float) { return (int)((b >> 23) & 0xff) - 127; }
__device__ __forceinline__ int exp_of_bits(unsigned long long b, double) { return (int)((b >> 52) & 0x7ff) - 1023; }
__device__ __forceinline__ unsigned long long abs_bits(float x) { return __float_as_uint(fabsf(x)); }
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(fabs(x));
}
template <typename R>
__device__ __forceinline__ R from_fix(long long v, int s);
template <>
__device__ __forceinline__ float from_fix<float>(long long v, int s) { return float_from_fix(v, s); }
template <>
__device__ __forceinline__ double from_fix<double>(long long v, int s) { return double_from_fix(v, s); }
__device__ __forceinline__ float rinv_real(float r, const ParamsDev& P) { return rinv_of(r, P.r_soft_f); }
__device__ __forceinline__ double rinv_real(double r, const ParamsDev& P) {
  const double rr = fmax(r, P.r_soft);
  return rr > 0.0 ? 1.0 / rr : 0.0;
}
__device__ __forceinline__ float phi_real(float M, float ri, float S, const ParamsDev& P) { return phi_of(M, ri, S, P.Gf); }
__device__ __forceinline__ double phi_real(double M, double ri, double S, const ParamsDev& P) {
  return __dmul_rn(-P.G, __fma_rn(M, ri, S));
}
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ bool neg(float x) { return signbit(x); }
__device__ __forceinline__ bool neg(double x) { return signbit(x); }

// All-FP64 recentring, written as the FP64 definition reads: d = x - c, then
// the minimum image, r^2 = (dx^2 + dy^2) + dz^2, r = sqrt(r^2) (both
// correctly rounded).
template <int CT>
__device__ __forceinline__ void offset_f64(const ParticlesDev& p, long long i, const HaloDev& H, double box,
                                           double d[3]) {
  double x[3];
  if (CT == AHF_COORD_F64) {
    x[0] = __ldg((const double*)p.x + i);
    x[1] = __ldg((const double*)p.y + i);
    x[2] = __ldg((const double*)p.z + i);
  } else {
    x[0] = (double)__ldg((const float*)p.x + i);
    x[1] = (double)__ldg((const float*)p.y + i);
    x[2] = (double)__ldg((const float*)p.z + i);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double v = __dsub_rn(x[a], H.c[a]);
    if (box > 0.0) {
      const double half = 0.5 * box;
      if (v > half) v = __dsub_rn(v, box);
      if (v < -half) v = __dadd_rn(v, box);
    }
    d[a] = v;
  }
}

__device__ __forceinline__ double r2_f64(const double d[3]) {
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

template <int CT>
__device__ __forceinline__ void load_velocity_f64(const ParticlesDev& p, long long i, double v[3]) {
  if (CT == AHF_COORD_F64) {
    v[0] = __ldg((const double*)p.vx + i);
    v[1] = __ldg((const double*)p.vy + i);
    v[2] = __ldg((const double*)p.vz + i);
  } else {
    v[0] = (double)__ldg((const float*)p.vx + i);
    v[1] = (double)__ldg((const float*)p.vy + i);
    v[2] = (double)__ldg((const float*)p.vz + i);
  }
}

template <int CT>
__device__ __forceinline__ double load_mass_f64(const ParticlesDev& p, long long i) {
  if (p.m == nullptr) return p.m0;
  if (CT == AHF_COORD_F64) return __ldg((const double*)p.m + i);
  return (double)__ldg((const float*)p.m + i);
}

// Member test, radius, mass and velocity of one candidate in precision R.
template <int CT>
__device__ __forceinline__ bool candidate(const ParticlesDev& p, long long pi, const HaloDev& H, const FrameDev& F,
                                          float& r, float& m, float v[3]) {
  long long f[3];
  float df[3];
  offset_of<CT>(p, pi, H, df, f);
  if (!member_of<CT>(p, pi, H, df, f)) return false;
  r = radius_of(df);
  m = load_mass<CT>(p, pi);
  load_velocity<CT>(p, pi, v);
  return true;
}
template <int CT>
__device__ __forceinline__ bool candidate(const ParticlesDev& p, long long pi, const HaloDev& H, const FrameDev& F,
                                          double& r, double& m, double v[3]) {
  double d[3];
  offset_f64<CT>(p, pi, H, F.box, d);
  const double r2 = r2_f64(d);
  if (!(r2 <= H.R2)) return false;
  r = sqrt(r2);
  m = load_mass_f64<CT>(p, pi);
  load_velocity_f64<CT>(p, pi, v);
  return true;
}

// w = v + H d of a member (the offset recomputed exactly as for its key).
template <int CT>
__device__ __forceinline__ void w_of(const ParticlesDev& p, long long pi, const HaloDev& H, const FrameDev& F,
                                     const ParamsDev& P, float w[3], float v[3], float& m) {
  long long f[3];
  float d[3];
  offset_of<CT>(p, pi, H, d, f);
  load_velocity<CT>(p, pi, v);
  m = load_mass<CT>(p, pi);
#pragma unroll
  for (int a = 0; a < 3; ++a) w[a] = fmaf(P.Hf, d[a], v[a]);
}
template <int CT>
__device__ __forceinline__ void w_of(const ParticlesDev& p, long long pi, const HaloDev& H, const FrameDev& F,
                                     const ParamsDev& P, double w[3], double v[3], double& m) {
  double d[3];
  offset_f64<CT>(p, pi, H, F.box, d);
  load_velocity_f64<CT>(p, pi, v);
  m = load_mass_f64<CT>(p, pi);
#pragma unroll
  for (int a = 0; a < 3; ++a) w[a] = __fma_rn(P.H, d[a], v[a]);
}
template <int CT>
__device__ __forceinline__ void velocity_real(const ParticlesDev& p, long long pi, float v[3]) {
  load_velocity<CT>(p, pi, v);
}
template <int CT>
__device__ __forceinline__ void velocity_real(const ParticlesDev& p, long long pi, double v[3]) {
  load_velocity_f64<CT>(p, pi, v);
}

// ---- prepare ---------------------------------------------------------------------

template <int CT, typename R>
__global__ void __launch_bounds__(T) g_prepare(GridLaunch L) {
  using Key = typename Prec<R>::Key;
  const int t = blockIdx.x;
  const int2 tr = L.tile_range[t];
  const int k = L.tile_halo[t];
  const HaloDev H = L.halos[k];
  const ParamsDev& P = L.prm;
  Key* key_a = (Key*)L.key_a;
  const Key NONMEMBER = ~(Key)0;
  Key orb = 0, andb = ~(Key)0;
  unsigned long long mxm = 0, mxr = 0, mxv = 0;
  int nmem = 0;
  for (int e = threadIdx.x; e < tr.y; e += T) {
    const long long g = (long long)tr.x + e;
    const long long i = g - H.gbase;                 // candidate position
    const long long slot = H.offset + i;
    long long pi = slot;
    bool ok = true;
    if (L.out.member_idx) {
      pi = L.out.member_idx[slot];
      if (pi < 0 || pi >= L.p.n) { ok = false; atomicOr(L.out.err, ERR_BAD_INDEX); }
    }
    Key key = NONMEMBER;
    if (ok) {
      R r, m, v[3];
      if (candidate<CT>(L.p, pi, H, L.frame, r, m, v)) {
        key = key_of(r);
        mxm = max(mxm, abs_bits(m));
        mxr = max(mxr, abs_bits(m * rinv_real(r, P)));
#pragma unroll
        for (int a = 0; a < 3; ++a) mxv = max(mxv, abs_bits(mul_rn(m, v[a])));
        ++nmem;
      }
    }
    if (key == NONMEMBER && L.out.removed_iter) L.out.removed_iter[slot] = -1;
    key_a[g] = key;
    L.val_a[g] = (uint32_t)i;
    orb |= key;
    andb &= key;
  }
  for (int o = 16; o > 0; o >>= 1) {
    orb |= __shfl_xor_sync(FULL_MASK, orb, o);
    andb &= __shfl_xor_sync(FULL_MASK, andb, o);
    mxm = max(mxm, __shfl_xor_sync(FULL_MASK, mxm, o));
    mxr = max(mxr, __shfl_xor_sync(FULL_MASK, mxr, o));
    mxv = max(mxv, __shfl_xor_sync(FULL_MASK, mxv, o));
  }
  nmem = __reduce_add_sync(FULL_MASK, nmem);
  if ((threadIdx.x & 31) == 0) {
    GridHaloState* st = L.state + k;
    atomicOr(&L.key_or_and[0], (unsigned long long)orb);
    atomicAnd(&L.key_or_and[1], (unsigned long long)andb | (Prec<R>::KEY_BYTES == 4 ? 0xffffffff00000000ull : 0ull));
    atomicMax(&st->mass_max_bits, mxm);
    atomicMax(&st->mr_max_bits, mxr);
    atomicMax(&st->mv_max_bits, mxv);
    if (nmem) atomicAdd((unsigned long long*)&st->n_member, (unsigned long long)nmem);
  }
}

template <typename R>
__global__ void g_scales(GridLaunch L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.n_halos) return;
  GridHaloState& s = L.state[k];
  const long long n = s.n_member;
  s.s_m = fix_scale(exp_of_bits(s.mass_max_bits, R()), n);
  s.s_mr = fix_scale(exp_of_bits(s.mr_max_bits, R()), n);
  s.s_mv = fix_scale(exp_of_bits(s.mv_max_bits, R()), n);
  s.n_alive = n;
  s.active = n > 0 ? 1 : 0;
  s.n_iter = 0;
  s.status = 0;
  s.part_iter = 0;
  s.band = 0;
  s.removed = 0;
  s.mv[0] = s.mv[1] = s.mv[2] = 0;
  s.k_first = 0x7fffffffffffffffll;
}

// ---- segmented radix sort ------------------------------------------------------------

// Tile histograms, stored per halo digit-major: the count of digit d in the
// halo's tile i (i = t - t0) sits at hist[256 t0 + d T_h + i], T_h the halo's
// tile count, so each digit's column over the halo's tiles is contiguous.
template <typename Key>
__global__ void __launch_bounds__(T) g_hist(const Key* __restrict__ key, const int2* __restrict__ tile_range,
                                            const int* __restrict__ tile_halo, const int* __restrict__ halo_tile0,
                                            uint32_t* __restrict__ tile_hist, int shift) {
  __shared__ uint32_t h[256];
  const int t = blockIdx.x;
  const int2 tr = tile_range[t];
  const int k = tile_halo[t];
  const int t0 = halo_tile0[k], th = halo_tile0[k + 1] - t0;
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < tr.y; e += T) atomicAdd(&h[(uint32_t)(key[tr.x + e] >> shift) & 0xffu], 1u);
  __syncthreads();
  tile_hist[(size_t)t0 * 256 + (size_t)threadIdx.x * th + (t - t0)] = h[threadIdx.x];
}

// One CTA per (halo, digit): exclusive prefix of the digit's counts over the
// halo's tiles (in place) and the digit's total.
__global__ void __launch_bounds__(256) g_digit_scan(uint32_t* __restrict__ tile_hist, const int* __restrict__ halo_tile0,
                                                    uint32_t* __restrict__ digit_base) {
  __shared__ uint32_t wt[8];
  __shared__ uint32_t carry;
  const int k = blockIdx.x >> 8, d = blockIdx.x & 255;
  const int t0 = halo_tile0[k], th = halo_tile0[k + 1] - t0;
  uint32_t* col = tile_hist + (size_t)t0 * 256 + (size_t)d * th;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < th; b += 256) {
    const int i = b + threadIdx.x;
    const uint32_t v = i < th ? col[i] : 0u;
    const uint32_t inc = warp_inclusive_scan(v, lane);
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    uint32_t base = carry;
    for (int w = 0; w < warp; ++w) base += wt[w];
    if (i < th) col[i] = base + inc - v;
    __syncthreads();
    if (threadIdx.x == 255) carry = base + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) digit_base[(size_t)k * 256 + d] = carry;
}

// One CTA per halo: digit totals -> first destination of each digit.
__global__ void __launch_bounds__(256) g_digit_base(uint32_t* __restrict__ digit_base) {
  __shared__ uint32_t wt[8];
  const int k = blockIdx.x, d = threadIdx.x, lane = d & 31, warp = d >> 5;
  const uint32_t v = digit_base[(size_t)k * 256 + d];
  const uint32_t inc = warp_inclusive_scan(v, lane);
  if (lane == 31) wt[warp] = inc;
  __syncthreads();
  uint32_t base = inc - v;
  for (int w = 0; w < warp; ++w) base += wt[w];
  digit_base[(size_t)k * 256 + d] = base;
}

template <typename Key>
__global__ void __launch_bounds__(T) g_scatter(const Key* __restrict__ kin, const uint32_t* __restrict__ vin,
                                               Key* __restrict__ kout, uint32_t* __restrict__ vout,
                                               const int2* __restrict__ tile_range, const int* __restrict__ tile_halo,
                                               const int* __restrict__ halo_tile0, const HaloDev* __restrict__ halos,
                                               const uint32_t* __restrict__ tile_off,
                                               const uint32_t* __restrict__ digit_base, int shift) {
  __shared__ uint16_t hist[NWARP * 256];
  __shared__ uint32_t doff[256];
  const int t = blockIdx.x;
  const int2 tr = tile_range[t];
  const int kh = tile_halo[t];
  const long long gb = halos[kh].gbase;
  const int t0 = halo_tile0[kh], th = halo_tile0[kh + 1] - t0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < NWARP * 256; i += T) hist[i] = 0;
  __syncthreads();
  constexpr int CH = TILE / NWARP;      // 256 elements per warp, 8 batches of 32
  Key key[IPT];
  uint32_t val[IPT];
  uint16_t rank[IPT];
#pragma unroll
  for (int b = 0; b < IPT; ++b) {
    const int e = warp * CH + b * 32 + lane;
    const bool valid = e < tr.y;
    key[b] = valid ? kin[tr.x + e] : (Key)0;
    val[b] = valid ? vin[tr.x + e] : 0u;
    const unsigned vmask = __ballot_sync(FULL_MASK, valid);
    rank[b] = 0;
    if (valid) {
      const uint32_t dg = (uint32_t)(key[b] >> shift) & 0xffu;
      const unsigned peers = __match_any_sync(vmask, dg);
      const unsigned below = peers & lanemask_lt();
      const uint16_t base = hist[warp * 256 + dg];
      rank[b] = (uint16_t)(base + __popc(below));
      __syncwarp(vmask);
      if (below == 0) hist[warp * 256 + dg] = (uint16_t)(base + __popc(peers));
    }
    __syncwarp();
  }
  __syncthreads();
  {
    // within-tile offsets of each (digit, warp) and the tile's global offsets
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < NWARP; ++w) {
      const uint32_t c = hist[w * 256 + d];
      hist[w * 256 + d] = (uint16_t)run;
      run += c;
    }
    doff[d] = digit_base[(size_t)kh * 256 + d] + tile_off[(size_t)t0 * 256 + (size_t)d * th + (t - t0)];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < IPT; ++b) {
    const int e = warp * CH + b * 32 + lane;
    if (e < tr.y) {
      const uint32_t dg = (uint32_t)(key[b] >> shift) & 0xffu;
      const long long dst = gb + (long long)doff[dg] + hist[warp * 256 + dg] + rank[b];
      kout[dst] = key[b];
      vout[dst] = val[b];
    }
  }
}

// ---- fill -------------------------------------------------------------------------

template <int CT, typename R>
__global__ void __launch_bounds__(T) g_fill(GridLaunch L) {
  using Key = typename Prec<R>::Key;
  using V4 = typename Prec<R>::V4;
  const Key* key = (const Key*)L.key_x;
  const uint32_t* val = L.val_x;
  V4* wm = (V4*)L.wm;
  R* rr = (R*)L.r;
  const int t = blockIdx.x;
  const int2 tr = L.tile_range[t];
  const int k = L.tile_halo[t];
  const HaloDev H = L.halos[k];
  const GridHaloState& S = L.state[k];
  const int s_v = S.s_mv;
  const long long nm = S.n_member;
  long long smv[3] = {0, 0, 0};
  for (int e = threadIdx.x; e < tr.y; e += T) {
    const long long g = (long long)tr.x + e;
    const long long p = g - H.gbase;
    if (p < nm) {
      const long long slot = H.offset + val[g];
      const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
      R w[3], v[3], m;
      w_of<CT>(L.p, pi, H, L.frame, L.prm, w, v, m);
      V4 q;
      q.x = w[0];
      q.y = w[1];
      q.z = w[2];
      q.w = m;
      wm[g] = q;
      rr[g] = real_of(key[g], R());
      if (L.uth) ((R*)L.uth)[g] = (R)(CT == AHF_COORD_F64 ? __ldg((const double*)L.p.u_th + pi)
                                                         : (double)__ldg((const float*)L.p.u_th + pi));
#pragma unroll
      for (int a = 0; a < 3; ++a) smv[a] += fix_real(mul_rn(m, v[a]), s_v);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long x = warp_sum(smv[a]);
    if ((threadIdx.x & 31) == 0 && x != 0)
      atomicAdd((unsigned long long*)&L.state[k].mv[a], (unsigned long long)x);
  }
}

// ---- iteration ------------------------------------------------------------------------

// Per tile: exact sums of m and m/r over alive members, and their count.
template <typename R>
__global__ void __launch_bounds__(T) g_tile_sums(GridLaunch L, int final_pass) {
  using V4 = typename Prec<R>::V4;
  const V4* wm = (const V4*)L.wm;
  const R* rr = (const R*)L.r;
  const int t = blockIdx.x;
  const int k = L.tile_halo[t];
  const GridHaloState& S = L.state[k];
  if (!final_pass && !S.active) return;
  const int2 tr = L.tile_range[t];
  const long long lim = L.halos[k].gbase + S.n_member;
  long long a = 0, b = 0, c = 0;
  const int s_m = S.s_m, s_r = S.s_mr;
  for (int e = threadIdx.x; e < tr.y; e += T) {
    const long long g = (long long)tr.x + e;
    if (g < lim) {
      const R m = wm[g].w;
      if (!neg(m)) {
        a += fix_real(m, s_m);
        b += fix_real(m * rinv_real(rr[g], L.prm), s_r);
        c += 1;
      }
    }
  }
  __shared__ long long red[NWARP][3];
  a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[warp][0] = a; red[warp][1] = b; red[warp][2] = c; }
  __syncthreads();
  if (threadIdx.x < 3) {
    long long s = 0;
    for (int w = 0; w < NWARP; ++w) s += red[w][threadIdx.x];
    L.tile_agg[(size_t)t * 3 + threadIdx.x] = s;
  }
}

// One CTA per halo: exclusive prefix of the tile sums, totals, v_bulk.
template <typename R>
__global__ void __launch_bounds__(256) g_tile_scan(GridLaunch L, int final_pass) {
  const int k = blockIdx.x;
  GridHaloState& S = L.state[k];
  if (!final_pass && !S.active) return;
  const int t0 = L.halo_tile0[k], t1 = L.halo_tile0[k + 1];
  __shared__ long long wt[8][3];
  __shared__ long long carry[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  for (int base = t0; base < t1; base += 256) {
    const int t = base + threadIdx.x;
    long long v[3] = {0, 0, 0};
    if (t < t1)
      for (int q = 0; q < 3; ++q) v[q] = L.tile_agg[(size_t)t * 3 + q];
    long long inc[3];
    for (int q = 0; q < 3; ++q) {
      inc[q] = warp_inclusive_scan(v[q], lane);
      if (lane == 31) wt[warp][q] = inc[q];
    }
    __syncthreads();
    for (int q = 0; q < 3; ++q) {
      long long b = carry[q];
      for (int w = 0; w < warp; ++w) b += wt[w][q];
      if (t < t1) L.tile_pre[(size_t)t * 3 + q] = b + inc[q] - v[q];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      long long s = 0;
      for (int w = 0; w < 8; ++w) s += wt[w][threadIdx.x];
      carry[threadIdx.x] += s;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    S.m_tot = carry[0];
    S.t_tot = carry[1];
    S.n_alive = carry[2];
    if (!final_pass) {
      // v_bulk of the current set (of the initial set with AHF_VAR_VBULK_INITIAL)
      if (S.n_iter == 0 || !L.prm.vbulk_initial) {
        if (sizeof(R) == 4) {
          const float mt = float_from_fix(carry[0], S.s_m);
          for (int a = 0; a < 3; ++a) S.vbulk[a] = float_from_fix(S.mv[a], S.s_mv) / mt;
        } else {
          const double mt = double_from_fix(carry[0], S.s_m);
          for (int a = 0; a < 3; ++a) S.vbulk_d[a] = double_from_fix(S.mv[a], S.s_mv) / mt;
        }
      }
      S.removed = 0;
      S.rem_m = 0;
      S.rem_mv[0] = S.rem_mv[1] = S.rem_mv[2] = 0;
      S.band_iter = 0;
    }
  }
}

// Blocked per-thread run inside a tile: exclusive prefix of the thread's
// first element from the tile prefix plus a block scan of thread totals.
struct TileScan {
  long long m, r, c;
};

__device__ __forceinline__ TileScan block_scan_tile(long long a, long long b, long long c, long long pre_a,
                                                     long long pre_b, long long pre_c) {
  __shared__ long long wt[NWARP][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long ia = warp_inclusive_scan(a, lane);
  const long long ib = warp_inclusive_scan(b, lane);
  const long long ic = warp_inclusive_scan(c, lane);
  if (lane == 31) { wt[warp][0] = ia; wt[warp][1] = ib; wt[warp][2] = ic; }
  __syncthreads();
  long long ba = pre_a, bb = pre_b, bc = pre_c;
  for (int w = 0; w < warp; ++w) { ba += wt[w][0]; bb += wt[w][1]; bc += wt[w][2]; }
  return TileScan{ba + ia - a, bb + ib - b, bc + ic - c};
}

template <int CT, typename R>
__global__ void __launch_bounds__(T) g_apply(GridLaunch L, int iter) {
  using V4 = typename Prec<R>::V4;
  V4* wm = (V4*)L.wm;
  const R* rr = (const R*)L.r;
  const int t = blockIdx.x;
  const int k = L.tile_halo[t];
  GridHaloState& S = L.state[k];
  if (!S.active) return;
  const int2 tr = L.tile_range[t];
  const HaloDev& H = L.halos[k];
  const long long lim = H.gbase + S.n_member;
  const int s_m = S.s_m, s_r = S.s_mr, s_v = S.s_mv;
  const ParamsDev& P = L.prm;
  R vb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) vb[a] = sizeof(R) == 4 ? (R)S.vbulk[a] : (R)S.vbulk_d[a];
  const R band = sizeof(R) == 4 ? (R)P.band_f : (R)P.band;
  const long long Ttot = S.t_tot;
  const long long g0 = (long long)tr.x + (long long)threadIdx.x * IPT;
  // pass 1: thread totals over its IPT consecutive elements
  V4 wmv[IPT];
  R rv[IPT];
  const R* uth = (const R*)L.uth;
  long long a = 0, b = 0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const long long g = g0 + q;
    const bool in = (threadIdx.x * IPT + q < tr.y) && g < lim;
    if (in) {
      wmv[q] = wm[g];
      rv[q] = rr[g];
    } else {
      wmv[q].x = wmv[q].y = wmv[q].z = (R)0;
      wmv[q].w = -(R)0;
      rv[q] = (R)1;
    }
    if (!neg(wmv[q].w)) {
      a += fix_real(wmv[q].w, s_m);
      b += fix_real(wmv[q].w * rinv_real(rv[q], P), s_r);
    }
  }
  TileScan ts = block_scan_tile(a, b, 0, L.tile_pre[(size_t)t * 3 + 0], L.tile_pre[(size_t)t * 3 + 1], 0);
  long long M = ts.m, Pp = ts.r;
  long long rm = 0, rv0 = 0, rv1 = 0, rv2 = 0;
  int nrem = 0, nband = 0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const R m = wmv[q].w;
    if (!neg(m)) {
      const R ri = rinv_real(rv[q], P);
      const long long mfix = fix_real(m, s_m);
      const long long rfix = fix_real(m * ri, s_r);
      const R phi = phi_real(from_fix<R>(M, s_m), ri, from_fix<R>(Ttot - Pp, s_r), P);
      const R ux = wmv[q].x - vb[0], uy = wmv[q].y - vb[1], uz = wmv[q].z - vb[2];
      R u2 = fma(uz, uz, fma(uy, uy, ux * ux));
      if (uth) u2 += (R)2 * uth[g0 + q];              // gas: |u|^2 + 2 u_th (Sect. 2.1)
      const R two_phi = (R)-2 * phi;
      if (fabs(u2 - two_phi) < band * two_phi) ++nband;
      if (u2 > two_phi) {
        const long long g = g0 + q;
        wm[g].w = -m;
        ++nrem;
        const long long slot = H.offset + L.val_x[g];
        const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
        R v[3];
        velocity_real<CT>(L.p, pi, v);
        rm += mfix;
        rv0 += fix_real(mul_rn(m, v[0]), s_v);
        rv1 += fix_real(mul_rn(m, v[1]), s_v);
        rv2 += fix_real(mul_rn(m, v[2]), s_v);
        if (L.out.removed_iter) L.out.removed_iter[slot] = iter;
      }
      M += mfix;
      Pp += rfix;
    }
  }
  nrem = __reduce_add_sync(FULL_MASK, nrem);
  nband = __reduce_add_sync(FULL_MASK, nband);
  if (__any_sync(FULL_MASK, nrem != 0)) {
    rm = warp_sum(rm); rv0 = warp_sum(rv0); rv1 = warp_sum(rv1); rv2 = warp_sum(rv2);
    if ((threadIdx.x & 31) == 0 && nrem) {
      atomicAdd((unsigned long long*)&S.rem_m, (unsigned long long)rm);
      atomicAdd((unsigned long long*)&S.rem_mv[0], (unsigned long long)rv0);
      atomicAdd((unsigned long long*)&S.rem_mv[1], (unsigned long long)rv1);
      atomicAdd((unsigned long long*)&S.rem_mv[2], (unsigned long long)rv2);
      atomicAdd((unsigned long long*)&S.removed, (unsigned long long)nrem);
    }
  }
  if ((threadIdx.x & 31) == 0 && nband) atomicAdd((unsigned long long*)&S.band_iter, (unsigned long long)nband);
}

__global__ void g_advance(GridLaunch L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.n_halos) return;
  GridHaloState& S = L.state[k];
  if (!S.active) return;
  S.n_iter += 1;
  S.part_iter += S.n_alive;
  S.band += S.band_iter;
  for (int a = 0; a < 3; ++a) S.mv[a] -= S.rem_mv[a];
  const long long left = S.n_alive - S.removed;
  if (S.removed == 0) {
    S.active = 0;
  } else if (left == 0) {
    S.active = 0;
    S.status |= AHF_HALO_EMPTY;
    S.n_alive = 0;
  } else if (S.n_iter >= L.prm.max_iter) {
    S.active = 0;
    S.status |= AHF_HALO_NOT_CONVERGED;
  }
  if (S.active) atomicAdd(L.any_active, 1);
}

// ---- finish ---------------------------------------------------------------------------

template <typename R>
__global__ void __launch_bounds__(T) g_emit(GridLaunch L) {
  using V4 = typename Prec<R>::V4;
  const V4* wm = (const V4*)L.wm;
  const R* rr = (const R*)L.r;
  R* rc = (R*)L.rc;
  const int t = blockIdx.x;
  const int k = L.tile_halo[t];
  GridHaloState& S = L.state[k];
  const int2 tr = L.tile_range[t];
  const HaloDev& H = L.halos[k];
  const long long lim = H.gbase + S.n_member;
  const int s_m = S.s_m, s_r = S.s_mr;
  const ParamsDev& P = L.prm;
  const long long Ttot = S.t_tot;
  const long long g0 = (long long)tr.x + (long long)threadIdx.x * IPT;
  R mq[IPT], rq[IPT];
  long long a = 0, b = 0, c = 0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const long long g = g0 + q;
    const bool in = (threadIdx.x * IPT + q < tr.y) && g < lim;
    mq[q] = in ? wm[g].w : -(R)0;
    rq[q] = in ? rr[g] : (R)1;
    if (!neg(mq[q])) {
      a += fix_real(mq[q], s_m);
      b += fix_real(mq[q] * rinv_real(rq[q], P), s_r);
      c += 1;
    }
  }
  const size_t tp = (size_t)t * 3;
  TileScan ts = block_scan_tile(a, b, c, L.tile_pre[tp], L.tile_pre[tp + 1], L.tile_pre[tp + 2]);
  long long M = ts.m, Pp = ts.r, C = ts.c;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const R m = mq[q];
    if (!neg(m)) {
      const long long g = g0 + q;
      const R ri = rinv_real(rq[q], P);
      const long long mfix = fix_real(m, s_m);
      const R phi = phi_real(from_fix<R>(M, s_m), ri, from_fix<R>(Ttot - Pp, s_r), P);
      const long long slot = H.offset + L.val_x[g];
      const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
      const long long dst = H.offset + C;
      L.out.bound_idx[dst] = pi;
      if (L.out.phi) ((R*)L.out.phi)[dst] = phi;
      if (L.out.removed_iter) L.out.removed_iter[slot] = 0;
      rc[H.gbase + C] = rq[q];
      L.mc[H.gbase + C] = M + mfix;
      M += mfix;
      Pp += fix_real(m * ri, s_r);
      C += 1;
    }
  }
}

// First compacted index k with M_k < delta_rho 4pi/3 r_{k+1}^3 (r_{N+1} = inf).
template <typename R>
__global__ void __launch_bounds__(T) g_virial(GridLaunch L) {
  const R* rc = (const R*)L.rc;
  const int t = blockIdx.x;
  const int k = L.tile_halo[t];
  GridHaloState& S = L.state[k];
  const int2 tr = L.tile_range[t];
  const long long gb = L.halos[k].gbase;
  const long long nb = S.n_alive;
  const ParamsDev& P = L.prm;
  long long kf = 0x7fffffffffffffffll;
  for (int e = threadIdx.x; e < tr.y; e += T) {
    const long long g = (long long)tr.x + e;
    const long long kk = g - gb;
    if (kk >= nb) break;
    bool cross = true;
    if (kk + 1 < nb) {
      const long long mk = L.mc[g];
      if (sizeof(R) == 4) {
        const float rn = (float)rc[g + 1];
        const float lhs = float_from_fix(mk, S.s_m);
        const float rhs = P.crit_f * rn * rn * rn;
        if (lhs < rhs * (1.0f - 1e-5f)) cross = true;
        else if (lhs > rhs * (1.0f + 1e-5f)) cross = false;
        else {
          const double rd = (double)rn;
          cross = double_from_fix(mk, S.s_m) < P.crit * rd * rd * rd;
        }
      } else {
        const double rd = (double)rc[g + 1];
        const double mkd = L.p.m == nullptr ? (double)(kk + 1) * L.p.m0 : double_from_fix(mk, S.s_m);
        cross = mkd < P.crit * rd * rd * rd;
      }
    }
    if (cross) { kf = kk; break; }
  }
  // warp min then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) kf = min(kf, __shfl_xor_sync(FULL_MASK, kf, o));
  if ((threadIdx.x & 31) == 0 && kf != 0x7fffffffffffffffll)
    atomicMin((unsigned long long*)&S.k_first, (unsigned long long)kf);
}

template <typename Real>
__global__ void g_result(GridLaunch L) {
  const Real* rc = (const Real*)L.rc;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.n_halos) return;
  const GridHaloState& S = L.state[k];
  const HaloDev& H = L.halos[k];
  ahf_result Rs;
  const long long nb = S.n_alive;
  Rs.n_bound = nb;
  Rs.n_member = S.n_member;
  Rs.part_iter = S.part_iter;
  Rs.n_band = S.band;
  Rs.n_iter = S.n_iter;
  Rs.k_vir = -1;
  Rs.m_vir = 0.0;
  Rs.r_vir = 0.0;
  int status = S.status;
  if (S.n_member == 0) status |= AHF_HALO_EMPTY;
  if (nb > 0) {
    const long long kk = S.k_first;
    // M_vir: (k+1) m0 in FP64 for a uniform mass, else the exact sum
    const bool unim = L.p.m == nullptr;
    const long long mkx = unim ? 0 : L.mc[H.gbase + kk];
    const double mk = unim ? double_from_fix(kk + 1, 0) * L.p.m0 : double_from_fix(mkx, S.s_m);
    if (kk == nb - 1) status |= AHF_HALO_RVIR_BEYOND_EDGE;
    bool none;
    if (sizeof(Real) == 4) {
      // the decision and the values as in the on-chip classes (the same bits)
      const float mkf = unim ? (float)(kk + 1) * L.p.m0f : float_from_fix(mkx, S.s_m);
      none = below_threshold(mk, mkf, (float)rc[H.gbase + kk], L.prm.crit_f, L.prm.crit);
    } else {
      const double rk = (double)rc[H.gbase + kk];
      none = mk < L.prm.crit * rk * rk * rk;
    }
    if (none) {
      status |= AHF_HALO_RVIR_NONE;
    } else {
      Rs.k_vir = kk;
      Rs.m_vir = mk;
      Rs.r_vir = virial_radius(mk, L.prm.inv_crit);
      if (L.prm.rise_edge && kk == nb - 1) {
        auto at = [&](long long k, double& r, double& m) {
          r = sizeof(Real) == 4 ? float_to_double((float)rc[H.gbase + k]) : (double)rc[H.gbase + k];
          m = unim ? double_from_fix(k + 1, 0) * L.p.m0 : double_from_fix(L.mc[H.gbase + k], S.s_m);
        };
        const long long ke = rise_edge_index(nb, at);
        if (ke >= 0) {
          at(ke, Rs.r_vir, Rs.m_vir);
          Rs.k_vir = ke;
          status |= AHF_HALO_RISE_EDGE;
        }
      }
    }
    const double mt = double_from_fix(S.m_tot, S.s_m);
    for (int a = 0; a < 3; ++a) Rs.vbulk[a] = quotient(double_from_fix(S.mv[a], S.s_mv), mt);
  } else {
    Rs.vbulk[0] = Rs.vbulk[1] = Rs.vbulk[2] = 0.0;
  }
  Rs.status = status;
  L.out.res[H.index] = Rs;
}

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

template <typename R>
cudaError_t prepare_t(const GridLaunch& L, cudaStream_t s) {
  if (L.p.coord_type == AHF_COORD_F64) g_prepare<AHF_COORD_F64, R><<<L.n_tiles, T, 0, s>>>(L);
  else g_prepare<AHF_COORD_F32_REL, R><<<L.n_tiles, T, 0, s>>>(L);
  g_scales<R><<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

template <typename Key>
cudaError_t sort_t(GridLaunch& L, cudaStream_t s, unsigned long long or_bits, unsigned long long and_bits) {
  const unsigned long long diff = or_bits ^ and_bits;
  Key *ki = (Key*)L.key_a, *ko = (Key*)L.key_b;
  uint32_t *vi = L.val_a, *vo = L.val_b;
  L.sort_passes = 0;
  for (int d = 0; d < (int)sizeof(Key); ++d) {
    if (!((diff >> (8 * d)) & 0xffull)) continue;
    ++L.sort_passes;
    const int shift = 8 * d;
    g_hist<Key><<<L.n_tiles, T, 0, s>>>(ki, L.tile_range, L.tile_halo, L.halo_tile0, L.tile_hist, shift);
    g_digit_scan<<<L.n_halos * 256, 256, 0, s>>>(L.tile_hist, L.halo_tile0, L.digit_base);
    g_digit_base<<<L.n_halos, 256, 0, s>>>(L.digit_base);
    g_scatter<Key><<<L.n_tiles, T, 0, s>>>(ki, vi, ko, vo, L.tile_range, L.tile_halo, L.halo_tile0, L.halos,
                                           L.tile_hist, L.digit_base, shift);
    Key* x = ki; ki = ko; ko = x;
    uint32_t* y = vi; vi = vo; vo = y;
  }
  L.key_x = ki;
  L.val_x = vi;
  return cudaGetLastError();
}

template <typename R>
cudaError_t fill_t(const GridLaunch& L, cudaStream_t s) {
  if (L.p.coord_type == AHF_COORD_F64) g_fill<AHF_COORD_F64, R><<<L.n_tiles, T, 0, s>>>(L);
  else g_fill<AHF_COORD_F32_REL, R><<<L.n_tiles, T, 0, s>>>(L);
  return cudaGetLastError();
}

template <typename R>
cudaError_t iterate_t(const GridLaunch& L, int iter, cudaStream_t s) {
  g_tile_sums<R><<<L.n_tiles, T, 0, s>>>(L, 0);
  g_tile_scan<R><<<L.n_halos, 256, 0, s>>>(L, 0);
  if (L.p.coord_type == AHF_COORD_F64) g_apply<AHF_COORD_F64, R><<<L.n_tiles, T, 0, s>>>(L, iter);
  else g_apply<AHF_COORD_F32_REL, R><<<L.n_tiles, T, 0, s>>>(L, iter);
  g_advance<<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

template <typename R>
cudaError_t finish_t(const GridLaunch& L, cudaStream_t s) {
  g_tile_sums<R><<<L.n_tiles, T, 0, s>>>(L, 1);
  g_tile_scan<R><<<L.n_halos, 256, 0, s>>>(L, 1);
  g_emit<R><<<L.n_tiles, T, 0, s>>>(L);
  g_virial<R><<<L.n_tiles, T, 0, s>>>(L);
  g_result<R><<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace

cudaError_t grid_prepare(const GridLaunch& L, cudaStream_t s) {
  return L.fp64 ? prepare_t<double>(L, s) : prepare_t<float>(L, s);
}

cudaError_t grid_sort(GridLaunch& L, cudaStream_t s, unsigned long long or_bits, unsigned long long and_bits) {
  return L.fp64 ? sort_t<unsigned long long>(L, s, or_bits, and_bits) : sort_t<uint32_t>(L, s, or_bits, and_bits);
}

cudaError_t grid_fill(const GridLaunch& L, cudaStream_t s) { return L.fp64 ? fill_t<double>(L, s) : fill_t<float>(L, s); }

cudaError_t grid_iterate(const GridLaunch& L, int iter, cudaStream_t s) {
  return L.fp64 ? iterate_t<double>(L, iter, s) : iterate_t<float>(L, iter, s);
}

cudaError_t grid_finish(const GridLaunch& L, cudaStream_t s) {
  return L.fp64 ? finish_t<double>(L, s) : finish_t<float>(L, s);
}

}  // namespace ahf
