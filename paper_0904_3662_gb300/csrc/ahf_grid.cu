// Multi-CTA class: haloes too large for one CTA's (or one cluster's) shared
// memory, and every halo in the all-FP64 mode.
//
// The haloes of this class share flat arrays (halo k owns [gbase_k,
// gbase_k + count_k)) cut into tiles of GRID_TILE elements that never cross
// a halo.  The steps are those of the on-chip classes (Sect. 2.1, Appendix
// A), laid out for HBM streaming:
//   prepare  one coalesced read of the candidates: recentring, sphere test,
//            radius key, and a 32-byte record per candidate, (w, r) and
//            (v, m) with w = v + H d (64 bytes in the all-FP64 mode)
//   sort     segmented stable LSD radix sort of (key, position) with 8-bit
//            digits (tile histograms, per-(halo, digit) scans over tiles,
//            digit bases, a scatter ranked by warp ballots and staged in
//            shared memory so that each digit's run is written contiguously);
//            the last pass gathers each member's record once and writes the
//            radial-order stream (w, r) (+ m), so no later step touches the
//            particle store
//   init     exact sums of the initial set per tile and per halo, v_bulk
//   passes   ONE streaming kernel per iteration: each tile takes the exact
//            prefix sums M(<r) and sum m/r of the tiles before it from the
//            tile prefixes of the current set, evaluates phi (Appendix A),
//            the escape test and the removals, and subtracts what it removed
//            from its own sums; the last tile of a halo to finish turns the
//            tiles' sums into the prefixes of the set left, the halo's
//            totals, v_bulk and its convergence
//   final    bound lists, phi, compacted radii and inclusive masses, the
//            first virial crossing, the records, and the profile rows by
//            binary search over the compacted radii
//
// No CTA ever waits for another one: a tile reads only prefixes that an
// earlier kernel finished, and each halo's bookkeeping is done by whichever
// of its tiles finishes last (an atomic count).

// Exact sums: long long fixed point in the mixed mode (the same scales and
// bits as the on-chip classes), __int128 in the all-FP64 mode, where a
// 64-bit quantum would limit large haloes to ~1e-11 relative in sum m/r.
#include <atomic>
#include <cstdint>

#include "ahf_device.cuh"

namespace ahf {
namespace {

constexpr int T = GRID_THREADS;         // 256
constexpr int TILE = GRID_TILE;         // 2048
constexpr int IPT = TILE / T;           // 8 elements per thread
constexpr int NWARP = T / 32;
static_assert(T == 256, "one thread per byte digit in the histograms and scans");

// Precision of the per-particle arithmetic.  float: the mixed mode (FP32
// radius key, FP32 phi and escape test).  double: the all-FP64 mode (FP64
// offsets, radius key, phi and escape test).
struct alignas(32) D4 {
  double x, y, z, w;
};
template <typename R>
struct Prec;
template <>
struct Prec<float> {
  using Key = uint32_t;
  using V4 = float4;
  using Acc = long long;
  static constexpr int ACC_BITS = 61;   // partial sums stay below 2^62
};
template <>
struct Prec<double> {
  using Key = unsigned long long;
  using V4 = D4;
  using Acc = __int128;
  static constexpr int ACC_BITS = 125;  // partial sums stay below 2^126
};

// ---- exact sums ---------------------------------------------------------------------

template <typename Acc>
__device__ __forceinline__ Acc& A(AccSlot& s) {
  return *reinterpret_cast<Acc*>(s.w);
}
template <typename Acc>
__device__ __forceinline__ Acc Ald(const AccSlot& s) {
  return *reinterpret_cast<const Acc*>(s.w);
}
// an AccSlot another CTA of the running kernel wrote (read through L2)
template <typename Acc>
__device__ __forceinline__ Acc Acg(const AccSlot& s);
template <>
__device__ __forceinline__ long long Acg<long long>(const AccSlot& s) {
  return __ldcg(&s.w[0]);
}
template <>
__device__ __forceinline__ __int128 Acg<__int128>(const AccSlot& s) {
  const unsigned long long lo = (unsigned long long)__ldcg(&s.w[0]);
  const unsigned long long hi = (unsigned long long)__ldcg(&s.w[1]);
  return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}

// Scale exponent s for sums of n terms of magnitude < 2^(emax+1) (the mixed
// mode's is fix_scale's).
template <typename R>
__device__ __forceinline__ int acc_scale(int emax, long long n) {
  int bits = 0;
  while (bits < 40 && (1ll << bits) < n) ++bits;
  return Prec<R>::ACC_BITS - bits - emax;
}

// round(x 2^s) for the all-FP64 mode (round half away from zero); the caller
// guarantees |x| 2^s < 2^126.
__device__ __forceinline__ __int128 fix128_from_double(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0;
  const long long mant = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = e - 1075 + s;
  __int128 v;
  if (sh >= 0) v = (__int128)mant << (sh > 73 ? 73 : sh);
  else if (sh > -54) v = (__int128)(((mant >> (-sh - 1)) + 1) >> 1);
  else v = 0;
  return (b >> 63) ? -v : v;
}

// v 2^-s as the nearest double (ties to even).
__device__ __forceinline__ double double_from_fix128(__int128 v, int s) {
  if (v == 0) return 0.0;
  const bool negv = v < 0;
  const unsigned __int128 a = negv ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  unsigned long long m;
  if (msb <= 52) {
    m = lo << (52 - msb);
  } else {
    const int sh = msb - 52;
    m = (unsigned long long)(a >> sh);
    const unsigned __int128 rem = a & (((unsigned __int128)1 << sh) - 1);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m == (1ull << 53)) {
        m >>= 1;
        ++msb;
      }
    }
  }
  // 2^msb (1 + frac): exact, msb <= 127
  const double d = __longlong_as_double((long long)(((unsigned long long)(msb + 1023) << 52) | (m & ((1ull << 52) - 1ull))));
  return scale_pow2d(negv ? -d : d, -s);
}

__device__ __forceinline__ long long fixr(float x, int s) { return fix_from_float(x, s); }
// round(x 2^s) for x >= 0 (the terms m and m/r): fix_from_float's value, with
// the round half up done as one add before the shift
__device__ __forceinline__ long long fixp(float x, int s) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)(b >> 23);
  if (e == 0) return 0;
  const int sh = e - 150 + s;
  const uint32_t mant = (b & 0x7fffffu) | 0x800000u;
  if (sh >= 0) return (long long)((unsigned long long)mant << (sh > 39 ? 39 : sh));
  const int rs = -sh;
  return rs > 24 ? 0ll : (long long)((mant + (1u << (rs - 1))) >> rs);
}
__device__ __forceinline__ __int128 fixp(double x, int s) { return fix128_from_double(x, s); }
__device__ __forceinline__ __int128 fixr(double x, int s) { return fix128_from_double(x, s); }
__device__ __forceinline__ float from_fix(long long v, int s, float) { return float_from_fix(v, s); }
__device__ __forceinline__ double from_fix(__int128 v, int s, double) { return double_from_fix128(v, s); }
__device__ __forceinline__ double dfix(long long v, int s) { return double_from_fix(v, s); }
__device__ __forceinline__ double dfix(__int128 v, int s) { return double_from_fix128(v, s); }

__device__ __forceinline__ uint32_t shfl_up_x(uint32_t x, int o) { return __shfl_up_sync(FULL_MASK, x, o); }
__device__ __forceinline__ int shfl_xor_x(int x, int o) { return __shfl_xor_sync(FULL_MASK, x, o); }
__device__ __forceinline__ long long shfl_up_x(long long x, int o) { return __shfl_up_sync(FULL_MASK, x, o); }
__device__ __forceinline__ __int128 shfl_up_x(__int128 x, int o) {
  const unsigned long long lo = __shfl_up_sync(FULL_MASK, (unsigned long long)x, o);
  const unsigned long long hi = __shfl_up_sync(FULL_MASK, (unsigned long long)((unsigned __int128)x >> 64), o);
  return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}
__device__ __forceinline__ long long shfl_xor_x(long long x, int o) { return __shfl_xor_sync(FULL_MASK, x, o); }
__device__ __forceinline__ __int128 shfl_xor_x(__int128 x, int o) {
  const unsigned long long lo = __shfl_xor_sync(FULL_MASK, (unsigned long long)x, o);
  const unsigned long long hi = __shfl_xor_sync(FULL_MASK, (unsigned long long)((unsigned __int128)x >> 64), o);
  return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}
__device__ __forceinline__ long long shfl_idx_x(long long x, int l) { return __shfl_sync(FULL_MASK, x, l); }
__device__ __forceinline__ __int128 shfl_idx_x(__int128 x, int l) {
  const unsigned long long lo = __shfl_sync(FULL_MASK, (unsigned long long)x, l);
  const unsigned long long hi = __shfl_sync(FULL_MASK, (unsigned long long)((unsigned __int128)x >> 64), l);
  return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}
template <typename X>
__device__ __forceinline__ X wsum(X x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += shfl_xor_x(x, o);
  return x;
}
template <typename X>
__device__ __forceinline__ X wscan(X x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const X y = shfl_up_x(x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Sum over the CTA of one value per thread (every thread gets the total).
template <typename X>
__device__ __forceinline__ X block_sum(X x, X* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = wsum(x);
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  X s = 0;
#pragma unroll
  for (int w = 0; w < NWARP; ++w) s += red[w];
  return s;
}

// block_sum for a CTA of NT threads.
template <typename X, int NT>
__device__ __forceinline__ X block_sum_n(X x, X* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = wsum(x);
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  X s = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}

// Exclusive prefix over the CTA's threads (thread order) of one value.
template <typename X>
__device__ __forceinline__ X block_excl(X x, X* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const X inc = wscan(x, lane);
  __syncthreads();
  if (lane == 31) red[warp] = inc;
  __syncthreads();
  X b = 0;
#pragma unroll
  for (int w = 0; w < NWARP; ++w)
    if (w < warp) b += red[w];
  return b + inc - x;
}

// ---- per-particle arithmetic ---------------------------------------------------------

__device__ __forceinline__ uint32_t key_of(float r) { return __float_as_uint(r); }
__device__ __forceinline__ unsigned long long key_of(double r) { return (unsigned long long)__double_as_longlong(r); }
__device__ __forceinline__ int exp_of_bits(unsigned long long b, float) { return (int)((b >> 23) & 0xff) - 127; }
__device__ __forceinline__ int exp_of_bits(unsigned long long b, double) { return (int)((b >> 52) & 0x7ff) - 1023; }
__device__ __forceinline__ unsigned long long abs_bits(float x) { return __float_as_uint(fabsf(x)); }
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(fabs(x));
}
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
__device__ __forceinline__ float fma_x(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_x(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float neg0(float) { return -0.0f; }
__device__ __forceinline__ double neg0(double) { return -0.0; }

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

// ---- prepare ---------------------------------------------------------------------

// The tile's counts of the keys' low byte, in g_hist's layout: the first radix
// pass sorts on that byte whenever it varies (it does for radii), and then
// reads these counts instead of running its own histogram kernel.
__device__ __forceinline__ void store_low_byte_hist(const GridLaunch& L, int t, int k, const uint32_t* h) {
  const int t0 = L.halo_tile0[k], th = L.halo_tile0[k + 1] - t0;
  L.tile_hist[(size_t)t0 * 256 + (size_t)threadIdx.x * th + (t - t0)] = h[threadIdx.x];
}

// The CTA's key range, per-halo maxima and member count merged into the call's
// words.  Every thread passes its warp's reduced values; the CTA reduces them
// once more and thread 0 issues an atomic only where it can change the word
// (OR, AND and max are idempotent, so a stale read costs an extra atomic,
// never a wrong value).  Thousands of tiles share a handful of words, so one
// atomic per warp and word would queue on the same addresses.
__device__ __forceinline__ void merge_prepare(const GridLaunch& L, int k, unsigned long long orb,
                                              unsigned long long andb, unsigned long long mxm,
                                              unsigned long long mxr, unsigned long long mxv, int nmem) {
  __shared__ unsigned long long red[5][NWARP];
  __shared__ int rn[NWARP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = orb;
    red[1][warp] = andb;
    red[2][warp] = mxm;
    red[3][warp] = mxr;
    red[4][warp] = mxv;
    rn[warp] = nmem;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned long long o = 0, a = ~0ull, m0 = 0, m1 = 0, m2 = 0;
  long long n = 0;
#pragma unroll
  for (int w = 0; w < NWARP; ++w) {
    o |= red[0][w];
    a &= red[1][w];
    m0 = max(m0, red[2][w]);
    m1 = max(m1, red[3][w]);
    m2 = max(m2, red[4][w]);
    n += rn[w];
  }
  GridHaloState* st = L.state + k;
  if (o & ~__ldcg(&L.ctl->key_or)) atomicOr(&L.ctl->key_or, o);
  if (~a & __ldcg(&L.ctl->key_and)) atomicAnd(&L.ctl->key_and, a);
  if (m0 > __ldcg(&st->mass_max_bits)) atomicMax(&st->mass_max_bits, m0);
  if (m1 > __ldcg(&st->mr_max_bits)) atomicMax(&st->mr_max_bits, m1);
  if (m2 > __ldcg(&st->mv_max_bits)) atomicMax(&st->mv_max_bits, m2);
  if (n) atomicAdd((unsigned long long*)&st->n_member, (unsigned long long)n);
}

// Mixed precision: the on-chip classes' float offsets (exact recentring),
// membership and radius; the record holds w = v + H d and r, then v and m.
template <int CT>
__global__ void __launch_bounds__(T, 4) g_prepare_mixed(GridLaunch L) {
  const int t = blockIdx.x;
  const int2 tr = L.tile_range[t];
  const int k = L.tile_halo[t];
  const HaloDev H = L.halos[k];
  const ParamsDev& P = L.prm;
  uint32_t* key_a = (uint32_t*)L.key_a;
  float4* rec = (float4*)L.rec;
  __shared__ uint32_t h0[256];
  h0[threadIdx.x] = 0u;
  Cand<CT> c[IPT];
  bool ok[IPT];
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int e = q * T + threadIdx.x;
    ok[q] = e < tr.y;
    if (ok[q]) {
      const long long slot = H.offset + ((long long)tr.x + e - H.gbase);
      long long pi = slot;
      if (L.out.member_idx) {
        pi = L.out.member_idx[slot];
        if (pi < 0 || pi >= L.p.n) {
          ok[q] = false;
          atomicOr(L.out.err, ERR_BAD_INDEX);
        }
      }
      if (ok[q]) load_cand<CT>(L.p, pi, c[q]);
    }
  }
  uint32_t orb = 0, andb = 0xffffffffu;
  unsigned long long mxm = 0, mxr = 0, mxv = 0;
  int nmem = 0;
  __syncthreads();                       // h0 zeroed
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int e = q * T + threadIdx.x;
    if (e >= tr.y) continue;
    const long long g = (long long)tr.x + e;
    uint32_t key = KEY_NONMEMBER;
    if (ok[q]) {
      float d[3];
      long long f[3];
      cand_offset<CT>(c[q], H, d, f);
      if (cand_member<CT>(c[q], H, d, f)) {
        const float r = radius_of(d);
        const float m = cand_mass<CT>(L.p, c[q]);
        float v[3];
        cand_velocity<CT>(c[q], v);
        rec[2 * g] = make_float4(fmaf(P.Hf, d[0], v[0]), fmaf(P.Hf, d[1], v[1]), fmaf(P.Hf, d[2], v[2]), r);
        rec[2 * g + 1] = make_float4(v[0], v[1], v[2], m);
        key = key_of(r);
        mxm = max(mxm, abs_bits(m));
        mxr = max(mxr, abs_bits(m * rinv_real(r, P)));
#pragma unroll
        for (int a = 0; a < 3; ++a) mxv = max(mxv, abs_bits(mul_rn(m, v[a])));
        ++nmem;
      }
    }
    if (L.out.removed_iter) L.out.removed_iter[H.offset + (g - H.gbase)] = key == KEY_NONMEMBER ? -1 : 0;
    key_a[g] = key;
    atomicAdd(&h0[key & 0xffu], 1u);
    orb |= key;
    andb &= key;
  }
  __syncthreads();
  store_low_byte_hist(L, t, k, h0);
  for (int o = 16; o > 0; o >>= 1) {
    orb |= __shfl_xor_sync(FULL_MASK, orb, o);
    andb &= __shfl_xor_sync(FULL_MASK, andb, o);
    mxm = max(mxm, __shfl_xor_sync(FULL_MASK, mxm, o));
    mxr = max(mxr, __shfl_xor_sync(FULL_MASK, mxr, o));
    mxv = max(mxv, __shfl_xor_sync(FULL_MASK, mxv, o));
  }
  nmem = __reduce_add_sync(FULL_MASK, nmem);
  merge_prepare(L, k, orb, (unsigned long long)andb | 0xffffffff00000000ull, mxm, mxr, mxv, nmem);
}

// All-FP64 mode: d = x - c in FP64 (minimum image), r^2 = (dx^2 + dy^2) + dz^2.
template <int CT>
__global__ void __launch_bounds__(T) g_prepare_f64(GridLaunch L) {
  const int t = blockIdx.x;
  const int2 tr = L.tile_range[t];
  const int k = L.tile_halo[t];
  const HaloDev H = L.halos[k];
  const ParamsDev& P = L.prm;
  unsigned long long* key_a = (unsigned long long*)L.key_a;
  D4* rec = (D4*)L.rec;
  unsigned long long orb = 0, andb = ~0ull, mxm = 0, mxr = 0, mxv = 0;
  int nmem = 0;
  __shared__ uint32_t h0[256];
  h0[threadIdx.x] = 0u;
  __syncthreads();
  for (int e = threadIdx.x; e < tr.y; e += T) {
    const long long g = (long long)tr.x + e;
    const long long slot = H.offset + (g - H.gbase);
    long long pi = slot;
    bool ok = true;
    if (L.out.member_idx) {
      pi = L.out.member_idx[slot];
      if (pi < 0 || pi >= L.p.n) {
        ok = false;
        atomicOr(L.out.err, ERR_BAD_INDEX);
      }
    }
    unsigned long long key = ~0ull;
    if (ok) {
      double d[3];
      offset_f64<CT>(L.p, pi, H, L.frame.box, d);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
      if (r2 <= H.R2) {
        const double r = sqrt(r2);
        const double m = load_mass_f64<CT>(L.p, pi);
        double v[3];
        load_velocity_f64<CT>(L.p, pi, v);
        D4 a, b;
        a.x = __fma_rn(P.H, d[0], v[0]);
        a.y = __fma_rn(P.H, d[1], v[1]);
        a.z = __fma_rn(P.H, d[2], v[2]);
        a.w = r;
        b.x = v[0];
        b.y = v[1];
        b.z = v[2];
        b.w = m;
        rec[2 * g] = a;
        rec[2 * g + 1] = b;
        key = key_of(r);
        mxm = max(mxm, abs_bits(m));
        mxr = max(mxr, abs_bits(m * rinv_real(r, P)));
#pragma unroll
        for (int q = 0; q < 3; ++q) mxv = max(mxv, abs_bits(mul_rn(m, v[q])));
        ++nmem;
      }
    }
    if (L.out.removed_iter) L.out.removed_iter[slot] = key == ~0ull ? -1 : 0;
    key_a[g] = key;
    atomicAdd(&h0[(uint32_t)key & 0xffu], 1u);
    orb |= key;
    andb &= key;
  }
  __syncthreads();
  store_low_byte_hist(L, t, k, h0);
  for (int o = 16; o > 0; o >>= 1) {
    orb |= __shfl_xor_sync(FULL_MASK, orb, o);
    andb &= __shfl_xor_sync(FULL_MASK, andb, o);
    mxm = max(mxm, __shfl_xor_sync(FULL_MASK, mxm, o));
    mxr = max(mxr, __shfl_xor_sync(FULL_MASK, mxr, o));
    mxv = max(mxv, __shfl_xor_sync(FULL_MASK, mxv, o));
  }
  nmem = __reduce_add_sync(FULL_MASK, nmem);
  merge_prepare(L, k, orb, andb, mxm, mxr, mxv, nmem);
}

template <typename R>
__global__ void g_scales(GridLaunch L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.n_halos) return;
  GridHaloState& s = L.state[k];
  const long long n = s.n_member;
  s.s_m = acc_scale<R>(exp_of_bits(s.mass_max_bits, R()), n);
  s.s_mr = acc_scale<R>(exp_of_bits(s.mr_max_bits, R()), n);
  s.s_mv = acc_scale<R>(exp_of_bits(s.mv_max_bits, R()), n);
  s.n_alive = n;
  s.active = 0;                          // set by the init pass
  s.n_iter = 0;
  s.status = 0;
  s.part_iter = 0;
  s.band = 0;
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

// Haloes of at most 256 tiles: one CTA per halo, thread d runs down digit
// d's column (exclusive prefix in place) and leaves the digit's total.
__global__ void __launch_bounds__(256) g_digit_scan_small(uint32_t* __restrict__ tile_hist,
                                                          const int* __restrict__ halo_tile0,
                                                          uint32_t* __restrict__ digit_base) {
  const int k = blockIdx.x, d = threadIdx.x;
  const int t0 = halo_tile0[k], th = halo_tile0[k + 1] - t0;
  if (th > 256) return;                  // g_digit_scan_big
  uint32_t* col = tile_hist + (size_t)t0 * 256 + (size_t)d * th;
  uint32_t run = 0;
  int i = 0;
  for (; i + 4 <= th; i += 4) {
    const uint32_t a = col[i], b = col[i + 1], c = col[i + 2], e = col[i + 3];
    col[i] = run;
    col[i + 1] = run + a;
    col[i + 2] = run + a + b;
    col[i + 3] = run + a + b + c;
    run += a + b + c + e;
  }
  for (; i < th; ++i) {
    const uint32_t a = col[i];
    col[i] = run;
    run += a;
  }
  digit_base[(size_t)k * 256 + d] = run;
}

// Haloes of more than 256 tiles: one CTA per (halo, digit) scans the column
// in chunks of 256 tiles.
__global__ void __launch_bounds__(256) g_digit_scan_big(uint32_t* __restrict__ tile_hist,
                                                        const int* __restrict__ halo_tile0,
                                                        const int* __restrict__ big, uint32_t* __restrict__ digit_base) {
  __shared__ uint32_t wt[8];
  __shared__ uint32_t carry;
  const int k = big[blockIdx.x >> 8], d = blockIdx.x & 255;
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

// Stable scatter of one tile by the digit at `shift`.  Each warp ranks its
// 8 batches of 32 keys by warp ballots on the digit's bits (the lanes with
// the same digit), the tile is re-ordered by digit in shared memory, and
// consecutive threads then write consecutive positions of each digit's run.
// FIRST: the values are the candidate positions (not read).  LAST: instead
// of (key, value) the radial-order streams are written from the records:
// (w, r), the mass (per-particle masses), u_th (gas) and the position; the
// tile's members' exact sum m v goes to tile_mv.
template <typename Key, typename R, bool FIRST, bool LAST>
__global__ void __launch_bounds__(T, LAST ? 3 : 5) g_scatter(GridLaunch L, const Key* __restrict__ kin,
                                               const uint32_t* __restrict__ vin, Key* __restrict__ kout,
                                               uint32_t* __restrict__ vout, int shift) {
  using V4 = typename Prec<R>::V4;
  using Acc = typename Prec<R>::Acc;
  __shared__ uint16_t whist[NWARP][256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t gofs[256];
  __shared__ uint32_t red[NWARP];
  __shared__ Key skey[TILE];
  __shared__ uint32_t sval[TILE];
  const int t = blockIdx.x;
  const int2 tr = L.tile_range[t];
  const int kh = L.tile_halo[t];
  const long long gb = L.halos[kh].gbase;
  const int t0 = L.halo_tile0[kh], th = L.halo_tile0[kh + 1] - t0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < NWARP * 256; i += T) (&whist[0][0])[i] = 0;
  // this tile's first global position of digit threadIdx.x (digit base + the
  // tiles before this one), loaded while the tile is ranked
  const uint32_t my_gofs =
      L.digit_base[(size_t)kh * 256 + threadIdx.x] + L.tile_hist[(size_t)t0 * 256 + (size_t)threadIdx.x * th + (t - t0)];
  constexpr int CH = TILE / NWARP;       // 256 elements per warp
  Key key[IPT];
  uint32_t val[IPT];
  uint16_t rank[IPT];
#pragma unroll
  for (int b = 0; b < IPT; ++b) {
    const int e = warp * CH + b * 32 + lane;
    const bool valid = e < tr.y;
    key[b] = valid ? kin[tr.x + e] : (Key)0;
    if (FIRST) val[b] = (uint32_t)((long long)tr.x + e - gb);
    else val[b] = valid ? vin[tr.x + e] : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < IPT; ++b) {
    const int e = warp * CH + b * 32 + lane;
    const bool valid = e < tr.y;
    const unsigned vmask = __ballot_sync(FULL_MASK, valid);
    const uint32_t dg = (uint32_t)(key[b] >> shift) & 0xffu;
    unsigned peers = vmask;
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const unsigned bb = __ballot_sync(FULL_MASK, (dg >> bit) & 1u);
      peers &= ((dg >> bit) & 1u) ? bb : ~bb;
    }
    const unsigned below = peers & lanemask_lt();
    uint16_t base = 0;
    if (valid) base = whist[warp][dg];
    rank[b] = (uint16_t)(base + __popc(below));
    __syncwarp();
    if (valid && below == 0) whist[warp][dg] = (uint16_t)(base + __popc(peers));
    __syncwarp();
  }
  __syncthreads();
  {
    // per digit: offsets of each warp's run, the digit's start in the tile
    // and its first global position (digit base + tiles before this one)
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
      const uint32_t c = whist[w][d];
      whist[w][d] = (uint16_t)run;
      run += c;
    }
    dstart[d] = block_excl(run, red);
    gofs[d] = my_gofs;
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < IPT; ++b) {
    const int e = warp * CH + b * 32 + lane;
    if (e < tr.y) {
      const uint32_t dg = (uint32_t)(key[b] >> shift) & 0xffu;
      const uint32_t lp = dstart[dg] + whist[warp][dg] + rank[b];
      skey[lp] = key[b];
      sval[lp] = val[b];
    }
  }
  __syncthreads();
  Acc smv[3] = {0, 0, 0};
  const int s_v = LAST ? L.state[kh].s_mv : 0;
  if (!LAST) {
    for (int i = threadIdx.x; i < tr.y; i += T) {
      const Key k = skey[i];
      const uint32_t dg = (uint32_t)(k >> shift) & 0xffu;
      const long long dst = gb + (long long)gofs[dg] + (i - (int)dstart[dg]);
      kout[dst] = k;
      vout[dst] = sval[i];
    }
  } else {
    // the records are gathered in batches of GB, every load of a batch issued
    // before its first use (the gathers are random within the halo)
    constexpr int GB = sizeof(R) == 4 ? 4 : 2;
    const V4* __restrict__ rec = (const V4*)L.rec;
#pragma unroll
    for (int b0 = 0; b0 < IPT; b0 += GB) {
      V4 ra[GB], rq[GB];
      uint32_t vv[GB];
      long long dd[GB];
      bool mem[GB];
#pragma unroll
      for (int j = 0; j < GB; ++j) {
        const int i = (b0 + j) * T + threadIdx.x;
        mem[j] = false;
        dd[j] = -1;
        if (i < tr.y) {
          const Key k = skey[i];
          vv[j] = sval[i];
          const uint32_t dg = (uint32_t)(k >> shift) & 0xffu;
          dd[j] = gb + (long long)gofs[dg] + (i - (int)dstart[dg]);
          mem[j] = k != ~(Key)0;
          if (mem[j]) {
            ra[j] = rec[2 * (gb + vv[j])];
            rq[j] = rec[2 * (gb + vv[j]) + 1];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < GB; ++j) {
        if (dd[j] < 0) continue;
        const long long dst = dd[j];
        L.val_x[dst] = vv[j];
        if (!mem[j]) continue;
        const V4 a = ra[j], q = rq[j];
        ((V4*)L.wr)[dst] = a;
        if (L.ms) ((R*)L.ms)[dst] = q.w;
        if (L.uth) {
          const long long slot = L.halos[kh].offset + vv[j];
          const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
          ((R*)L.uth)[dst] = (R)(L.p.coord_type == AHF_COORD_F64 ? __ldg((const double*)L.p.u_th + pi)
                                                                 : (double)__ldg((const float*)L.p.u_th + pi));
        }
        smv[0] += fixr(mul_rn(q.w, q.x), s_v);
        smv[1] += fixr(mul_rn(q.w, q.y), s_v);
        smv[2] += fixr(mul_rn(q.w, q.z), s_v);
      }
    }
  }
  if (LAST) {
    __shared__ Acc racc[NWARP];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const Acc s = block_sum(smv[a], racc);
      if (threadIdx.x == 0) A<Acc>(L.tile_mv[3 * (size_t)t + a]) = s;
    }
  }
}

// No radix pass (every key equal): the radial order is the candidate order.
template <typename R>
__global__ void __launch_bounds__(T) g_fill_identity(GridLaunch L) {
  using V4 = typename Prec<R>::V4;
  using Key = typename Prec<R>::Key;
  using Acc = typename Prec<R>::Acc;
  const int t = blockIdx.x;
  const int2 tr = L.tile_range[t];
  const int kh = L.tile_halo[t];
  const long long gb = L.halos[kh].gbase;
  const int s_v = L.state[kh].s_mv;
  const Key* key = (const Key*)L.key_a;
  Acc smv[3] = {0, 0, 0};
  for (int e = threadIdx.x; e < tr.y; e += T) {
    const long long g = (long long)tr.x + e;
    const uint32_t v = (uint32_t)(g - gb);
    L.val_x[g] = v;
    if (key[g] != ~(Key)0) {
      const V4* rc = (const V4*)L.rec + 2 * g;
      const V4 a = rc[0], q = rc[1];
      ((V4*)L.wr)[g] = a;
      if (L.ms) ((R*)L.ms)[g] = q.w;
      if (L.uth) {
        const long long slot = L.halos[kh].offset + v;
        const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
        ((R*)L.uth)[g] = (R)(L.p.coord_type == AHF_COORD_F64 ? __ldg((const double*)L.p.u_th + pi)
                                                             : (double)__ldg((const float*)L.p.u_th + pi));
      }
      smv[0] += fixr(mul_rn(q.w, q.x), s_v);
      smv[1] += fixr(mul_rn(q.w, q.y), s_v);
      smv[2] += fixr(mul_rn(q.w, q.z), s_v);
    }
  }
  __shared__ Acc racc[NWARP];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Acc s = block_sum(smv[a], racc);
    if (threadIdx.x == 0) A<Acc>(L.tile_mv[3 * (size_t)t + a]) = s;
  }
}

// ---- sub-tiles: the unit of a pass -------------------------------------------------------

// Sub-tile u covers elements [(u % SPT) SUB, (u % SPT + 1) SUB) of tile u / SPT
// (clipped to the tile); one warp handles it, element j of row i at position
// 32 i + lane, so that each row is one coalesced access.
constexpr int SUB = GRID_SUB;           // 256
constexpr int SPT = TILE / SUB;         // 8 sub-tiles per tile
constexpr int ROWS = SUB / 32;          // 8
constexpr int HT_BIG = 1024;            // threads of the per-halo kernel (largest halo > 64 tiles)
constexpr int HT_SMALL = 256;           // (otherwise)

// True once a pass of this call gave up waiting for a tensor copy: the
// sums it left are incomplete, so every later kernel of the class skips its
// work (the call's outputs are undefined and ahf_sync reports the timeout).
__device__ __forceinline__ bool gave_up(const GridLaunch& L) { return (__ldcg(L.out.err) & ERR_TIMEOUT) != 0; }

// Atomic add of an exact sum into a slot (the __int128 one from two 64-bit
// atomics: the low word's carry goes into the high word, so the total is
// exact once every addition has landed).
__device__ __forceinline__ void atomic_acc(AccSlot& s, long long v) {
  atomicAdd((unsigned long long*)&s.w[0], (unsigned long long)v);
}
__device__ __forceinline__ void atomic_acc(AccSlot& s, __int128 v) {
  const unsigned long long lo = (unsigned long long)v;
  const unsigned long long hi = (unsigned long long)((unsigned __int128)v >> 64);
  const unsigned long long old = atomicAdd((unsigned long long*)&s.w[0], lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  atomicAdd((unsigned long long*)&s.w[1], hi + carry);
}

// v_bulk = sum m v / sum m of the current set, into the halo state.
template <typename R>
__device__ __forceinline__ void set_vbulk(GridHaloState& S, typename Prec<R>::Acc m,
                                          const typename Prec<R>::Acc mv[3]) {
  if (sizeof(R) == 4) {
    const float mt = from_fix(m, S.s_m, R());
    for (int a = 0; a < 3; ++a) S.vbulk[a] = (float)from_fix(mv[a], S.s_mv, R()) / mt;
  } else {
    const double mt = dfix(m, S.s_m);
    for (int a = 0; a < 3; ++a) S.vbulk_d[a] = dfix(mv[a], S.s_mv) / mt;
  }
}

// x 2^-s from an exact sum: in the mixed mode float_from_fix's bits, with
// 2^-s passed as a float (0 when it is not a normal float: then the general
// route); in the FP64 mode the nearest double.
__device__ __forceinline__ float fix_to_real(long long v, int s, float sc, float) {
  if (sc == 0.0f) return float_from_fix(v, s);
  const float hi = (float)(int)(v >> 32);
  const float lo = (float)(unsigned)(v & 0xffffffffll);
  return fmaf(hi, 4294967296.0f, lo) * sc;
}
__device__ __forceinline__ double fix_to_real(__int128 v, int s, float, double) { return double_from_fix128(v, s); }

// Sums of the initial set (all members alive) per sub-tile, one warp each,
// into copy 1 (the first pass's).
template <typename R>
__global__ void __launch_bounds__(T) g_sums(GridLaunch L) {
  using V4 = typename Prec<R>::V4;
  using Acc = typename Prec<R>::Acc;
  const int lane = threadIdx.x & 31;
  const int n_sub = L.n_tiles * SPT;
  const int u = (blockIdx.x * T + threadIdx.x) >> 5;     // one warp per sub-tile
  if (u >= n_sub) return;
  const V4* wr = (const V4*)L.wr;
  const R* ms = (const R*)L.ms;
  const R m0 = sizeof(R) == 4 ? (R)L.p.m0f : (R)L.p.m0;
  const int t = u / SPT;
  const int2 tr = L.tile_range[t];
  const int e0 = (u % SPT) * SUB;
  // the rows are read before the halo's state arrives (the loads depend on
  // the tile only); elements past the last member are dropped afterwards
  R rq[ROWS], mq[ROWS];
#pragma unroll
  for (int i = 0; i < ROWS; ++i) {
    const int e = e0 + 32 * i + lane;
    const long long g = (long long)tr.x + e;
    rq[i] = e < tr.y ? wr[g].w : (R)0;
    mq[i] = (e < tr.y && ms) ? ms[g] : m0;
  }
  const int k = L.tile_halo[t];
  const GridHaloState& S = L.state[k];
  const long long lim = L.halos[k].gbase + S.n_member;
  Acc a = 0, b = 0;
  int c = 0;
#pragma unroll
  for (int i = 0; i < ROWS; ++i) {
    const int e = e0 + 32 * i + lane;
    const long long g = (long long)tr.x + e;
    if (e < tr.y && g < lim) {
      a += fixp(mq[i], S.s_m);
      b += fixp(mq[i] * rinv_real(rq[i], L.prm), S.s_mr);
      ++c;
    }
  }
  a = wsum(a);
  b = wsum(b);
  c = __reduce_add_sync(FULL_MASK, c);
  if (lane == 0) {
    ((Acc*)L.agg_m)[n_sub + u] = a;
    ((Acc*)L.agg_r)[n_sub + u] = b;
    L.agg_c[n_sub + u] = c;
  }
}

// Per halo, after the initial sums (INIT, pass 0) or after pass `pass`: the
// tiles' sums of the set left (copy (pass + 1) & 1 of the sub-tile sums),
// their exclusive prefix over the halo (for the next pass and the final one),
// the totals, and the halo's bookkeeping: iterations, particle-iterations,
// band tests, sum m v, v_bulk, convergence (Sect. 2.1, Appendix A: the loop
// ends when an iteration removes nothing).  Each thread takes a run of
// consecutive tiles; the runs' sums are scanned over the CTA.
// The sub-tiles of the haloes still active are listed for the next pass.
template <typename R, bool INIT, int HT>
__global__ void __launch_bounds__(HT) g_halo(GridLaunch L, int pass) {
  if (gave_up(L)) return;
  using Acc = typename Prec<R>::Acc;
  constexpr int CH = 1024;                 // tiles per chunk held in shared memory
  constexpr int NW = HT / 32;
  __shared__ Acc racc[NW];
  __shared__ Acc wm_[NW], wr_[NW];
  __shared__ long long wc_[NW];
  __shared__ Acc tm_[CH], tr_[CH];
  __shared__ long long tc_[CH];
  __shared__ int s_nw;
  __shared__ Acc s_tm, s_tr;
  __shared__ long long s_tc;
  __shared__ float s_vb[3];                // the skip test's halo input
  __shared__ int s_wn[NW], s_wb[NW];       // kept sub-tiles per warp, their list positions
  __shared__ int s_kept;                   // sub-tiles of the halo on the next list
  const int k = blockIdx.x;
  GridHaloState& S = L.state[k];
  if (!INIT && !S.active) return;
  const int n_sub = L.n_tiles * SPT;
  const int cp = (pass + 1) & 1;
  const Acc* am = (const Acc*)L.agg_m + (size_t)cp * n_sub;
  const Acc* ar = (const Acc*)L.agg_r + (size_t)cp * n_sub;
  const int* ac = L.agg_c + (size_t)cp * n_sub;
  Acc* pm = (Acc*)L.pre_m;
  Acc* pr = (Acc*)L.pre_r;
  const int t0 = L.halo_tile0[k], t1 = L.halo_tile0[k + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // only the sub-tiles holding members carry sums (the others are never
  // written by a pass)
  const int u_end = t0 * SPT + (int)((S.n_member + SUB - 1) / SUB);
  Acc cm = 0, cr = 0;                      // carry: the sums of the chunks before
  long long cc = 0;
  for (int c0 = t0; c0 < t1; c0 += CH) {
    const int cn = min(CH, t1 - c0);
    // tile sums, SPT lanes per tile (coalesced), reduced by shuffles; the
    // chunk's loads (CH * SPT / HT per thread) go out together
    constexpr int LPT = 8;
    for (int xr = 0; xr < cn * SPT; xr += LPT * HT) {
    Acc lm[LPT], lr[LPT];
    int lc[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      const int x = xr + q * HT + threadIdx.x;
      const int u = c0 * SPT + x;
      const bool in = x < cn * SPT && u < u_end;
      lm[q] = in ? am[u] : (Acc)0;
      lr[q] = in ? ar[u] : (Acc)0;
      lc[q] = in ? ac[u] : 0;
    }
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      const int x = xr + q * HT + threadIdx.x;
      Acc m = lm[q], r = lr[q];
      int c = lc[q];
#pragma unroll
      for (int o = 1; o < SPT; o <<= 1) {
        m += shfl_xor_x(m, o);
        r += shfl_xor_x(r, o);
        c += shfl_xor_x(c, o);
      }
      if ((x % SPT) == 0 && x < cn * SPT) {
        tm_[x / SPT] = m;
        tr_[x / SPT] = r;
        tc_[x / SPT] = c;
      }
    }
    }
    __syncthreads();
    // exclusive scan of the chunk's tile sums: a run of consecutive tiles per thread
    const int per = (cn + HT - 1) / HT;
    const int j0 = min(cn, (int)threadIdx.x * per), j1 = min(j0 + per, cn);
    Acc sm = 0, sr = 0;
    long long sc = 0;
    for (int j = j0; j < j1; ++j) {
      sm += tm_[j];
      sr += tr_[j];
      sc += tc_[j];
    }
    const Acc im = wscan(sm, lane), ir = wscan(sr, lane);
    const long long ic = wscan(sc, lane);
    if (lane == 31) {
      wm_[warp] = im;
      wr_[warp] = ir;
      wc_[warp] = ic;
    }
    __syncthreads();
    if (warp == 0) {
      const bool in = lane < NW;
      const Acc xm = in ? wm_[lane] : (Acc)0, xr = in ? wr_[lane] : (Acc)0;
      const long long xc = in ? wc_[lane] : 0ll;
      const Acc ym = wscan(xm, lane), yr = wscan(xr, lane);
      const long long yc = wscan(xc, lane);
      __syncwarp();
      if (in) {
        wm_[lane] = ym - xm;
        wr_[lane] = yr - xr;
        wc_[lane] = yc - xc;
      }
      if (lane == 31) {
        s_tm = ym;
        s_tr = yr;
        s_tc = yc;
      }
    }
    __syncthreads();
    Acc em = cm + wm_[warp] + im - sm, er = cr + wr_[warp] + ir - sr;
    long long ec = cc + wc_[warp] + ic - sc;
    for (int j = j0; j < j1; ++j) {
      pm[c0 + j] = em;
      pr[c0 + j] = er;
      L.pre_c[c0 + j] = ec;
      em += tm_[j];
      er += tr_[j];
      ec += tc_[j];
    }
    cm += s_tm;
    cr += s_tr;
    cc += s_tc;
    __syncthreads();                       // the chunk's shared arrays are reused
  }
  const Acc M = cm, Rr = cr;
  const long long C = cc;
  Acc mvs[3] = {0, 0, 0};
  if (INIT) {
    // sum m v of the members, from the sort's per-tile sums
    for (int j = t0 + threadIdx.x; j < t1; j += HT)
#pragma unroll
      for (int q = 0; q < 3; ++q) mvs[q] += Ald<Acc>(L.tile_mv[3 * (size_t)j + q]);
#pragma unroll
    for (int q = 0; q < 3; ++q) mvs[q] = block_sum_n<Acc, HT>(mvs[q], racc);
  }
  if (threadIdx.x == 0) {
    Acc mv[3];
    int active;
    if (INIT) {
#pragma unroll
      for (int q = 0; q < 3; ++q) mv[q] = mvs[q];
      active = C > 0 ? 1 : 0;
    } else {
      const long long alive = S.n_alive;
      S.part_iter += alive;
      S.band += S.band_pass;
      S.band_pass = 0;
      S.n_iter = pass;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        mv[q] = Ald<Acc>(S.mv[q]) - Ald<Acc>(S.rem_mv[q]);
        A<Acc>(S.rem_mv[q]) = 0;
      }
      active = 1;
      if (C == alive) {
        active = 0;
      } else if (C == 0) {
        active = 0;
        S.status |= AHF_HALO_EMPTY;
      } else if (pass >= L.prm.max_iter) {
        active = 0;
        S.status |= AHF_HALO_NOT_CONVERGED;
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) A<Acc>(S.mv[q]) = mv[q];
    A<Acc>(S.m_tot) = M;
    A<Acc>(S.t_tot) = Rr;
    S.n_alive = C;
    if (active && (INIT || !L.prm.vbulk_initial)) set_vbulk<R>(S, M, mv);
    S.active = active;
    // the mass lost so far (exact sums), for the skip records and test
    if (INIT) A<Acc>(S.m_init) = M;
    S.mrem = INIT ? 0.0 : dfix(Ald<Acc>(S.m_init) - M, S.s_m);
#pragma unroll
    for (int q = 0; q < 3; ++q) s_vb[q] = sizeof(R) == 4 ? S.vbulk[q] : (float)S.vbulk_d[q];
    // the halo's sub-tiles holding members go on the next pass's list
    s_nw = active ? (int)((S.n_member + SUB - 1) / SUB) : 0;
    s_kept = 0;
  }
  __syncthreads();
  const int nw = s_nw;
  if (nw) {
    const long long nm = S.n_member, gb = L.halos[k].gbase;
    int* wn = &L.ctl->work_n[(pass + 1) & 1];
    int4* list = L.work + (size_t)((pass + 1) & 1) * n_sub;
    const double mrem = S.mrem;
    const float vb0 = s_vb[0], vb1 = s_vb[1], vb2 = s_vb[2];
    const float two_g = 2.0f * L.prm.Gf, rsoft = L.prm.r_soft_f;
    // RB sub-tiles per thread and round, their records loaded together
    constexpr int RB = 4;
    for (int j0 = 0; j0 < nw; j0 += RB * HT) {
      bool keep[RB];
      SkipRec rc[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int j = j0 + r * HT + threadIdx.x;
        keep[r] = j < nw;
        if (!INIT && keep[r]) rc[r] = L.skip[t0 * SPT + j];
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int j = j0 + r * HT + threadIdx.x;
        const int u = t0 * SPT + j;
        if (INIT || !keep[r]) continue;
        // a sub-tile tested in an earlier pass stays out while its members
        // can neither be removed nor fall in the band: since that test each
        // member's 2|phi| fell by at most 2 G dM / max(r, r_soft) (the
        // halo lost mass dM, each removed particle's term at most m / r of
        // the member's own radius), and its |u|^2 rose by at most
        // 2 |u| dv + dv^2 (v_bulk moved by dv); the record's margin (slack
        // 2^-16 of 2|phi| for the float rounding of both tests) must exceed
        // that, with 2^-10 more on the bound for its own rounding
        const float dm = (float)(mrem - rc[r].mrem) * (1.0f + 0x1p-20f);
        const float reff = fmaxf(rc[r].rin, rsoft);
        const float ax = vb0 - rc[r].vb[0], ay = vb1 - rc[r].vb[1], az = vb2 - rc[r].vb[2];
        const float vmag = fabsf(vb0) + fabsf(vb1) + fabsf(vb2) + fabsf(rc[r].vb[0]) + fabsf(rc[r].vb[1]) +
                           fabsf(rc[r].vb[2]);
        const float dv = sqrtf(fmaf(az, az, fmaf(ay, ay, ax * ax))) * (1.0f + 0x1p-20f) + vmag * 0x1p-20f;
        const float bound = (two_g * dm / reff + dv * fmaf(2.0f, rc[r].umax, dv)) * (1.0f + 0x1p-10f);
        if (reff > 0.0f && isfinite(bound) && rc[r].margin > bound) {
          keep[r] = false;
          // its sums carry over to the copy the next pass would have written
          const size_t a = (size_t)((pass + 1) & 1) * n_sub + u, b = (size_t)(pass & 1) * n_sub + u;
          ((Acc*)L.agg_m)[b] = ((const Acc*)L.agg_m)[a];
          ((Acc*)L.agg_r)[b] = ((const Acc*)L.agg_r)[a];
          L.agg_c[b] = L.agg_c[a];
        }
      }
      // list positions: a warp scan of the warps' counts, one reservation per round
      unsigned bal[RB];
      int cnt = 0;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        bal[r] = __ballot_sync(FULL_MASK, keep[r]);
        cnt += __popc(bal[r]);
      }
      if (lane == 0) s_wn[warp] = cnt;
      __syncthreads();
      if (warp == 0) {
        const int x = lane < NW ? s_wn[lane] : 0;
        const int inc = (int)wscan((uint32_t)x, lane);
        int base = 0;
        if (lane == 31 && inc) base = atomicAdd(wn, inc);
        base = __shfl_sync(FULL_MASK, base, 31);
        if (lane < NW) s_wb[lane] = base + inc - x;
        if (lane == 31) s_kept += inc;
      }
      __syncthreads();
      int off = s_wb[warp];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int j = j0 + r * HT + threadIdx.x;
        if (keep[r])
          list[off + __popc(bal[r] & lanemask_lt())] =
              make_int4(t0 * SPT + j, k, (int)(gb + (long long)j * SUB), (int)min((long long)SUB, nm - (long long)j * SUB));
        off += __popc(bal[r]);
      }
      __syncthreads();                     // s_wn, s_wb are reused
    }
    // every sub-tile left out: the next pass would remove nothing, so the
    // halo converges there (its particle-iterations counted, no band tests)
    if (!INIT && threadIdx.x == 0 && s_kept == 0) {
      S.part_iter += S.n_alive;
      S.n_iter = pass + 1;
      S.active = 0;
    }
  }
}

// ---- one unbinding pass -----------------------------------------------------------------

constexpr int EPL = SUB / 32;            // 8 consecutive elements per lane

// Prefix sums of a sub-tile's start: the tile's prefix plus the sums of the
// tile's sub-tiles before it in copy `cp` (lanes < u % SPT read one each).
template <typename Acc>
__device__ __forceinline__ void sub_prefix(const GridLaunch& L, int u, int t, int cp, Acc& M, Acc& P, long long* C) {
  const int lane = threadIdx.x & 31;
  const int n_sub = L.n_tiles * SPT;
  const int ui = u % SPT;
  Acc m = 0, r = 0;
  int c = 0;
  if (lane < ui) {
    const size_t j = (size_t)cp * n_sub + (u - ui) + lane;
    m = ((const Acc*)L.agg_m)[j];
    r = ((const Acc*)L.agg_r)[j];
    if (C) c = L.agg_c[j];
  }
  M = ((const Acc*)L.pre_m)[t] + wsum(m);
  P = ((const Acc*)L.pre_r)[t] + wsum(r);
  if (C) *C = L.pre_c[t] + __reduce_add_sync(FULL_MASK, c);
}

// The skip record of sub-tile u from the lanes' margins and |u|^2 maxima
// (lane 0's first element is the sub-tile's first: its |r| bounds the
// members' radii from below); conservative roundings to float.
template <typename R>
__device__ __forceinline__ void write_skip(const GridLaunch& L, int u, const GridHaloState& S, R mg, R uu, R r0,
                                           const R vb[3]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mg = fmin(mg, __shfl_xor_sync(FULL_MASK, mg, o));
    uu = fmax(uu, __shfl_xor_sync(FULL_MASK, uu, o));
  }
  if ((threadIdx.x & 31) != 0) return;
  SkipRec rc;
  if (sizeof(R) == 4) {
    rc.margin = (float)mg;
    rc.umax = __fsqrt_ru((float)uu);
    rc.rin = fabsf((float)r0);
  } else {
    rc.margin = __double2float_rd((double)mg);
    rc.umax = __double2float_ru(sqrt((double)uu));
    rc.rin = __double2float_rd(fabs((double)r0));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) rc.vb[a] = (float)vb[a];
  rc.mrem = S.mrem;
  L.skip[u] = rc;
}

// Phi and the escape test over sub-tile w.x (halo w.y) in pass `pass`, by
// one warp: lane l holds elements [8 l, 8 l + 8) of the sub-tile; one warp
// scan of the lanes' sums places every element's prefix.  The pass only
// decides: it leaves the sub-tile's sums after the removals for the next
// pass and one byte of removal flags per lane; g_removed does the rest.
// FAST: the scales 2^-s of the halo are normal floats (the conversions of
// the exact sums to float are then a multiply; same bits).
template <typename R, bool UNIF, bool GAS, bool FAST>
__device__ __forceinline__ void pass_sub(const GridLaunch& L, const int4 w, int pass) {
  using V4 = typename Prec<R>::V4;
  using Acc = typename Prec<R>::Acc;
  const int u = w.x, k = w.y, t = u / SPT;
  GridHaloState& S = L.state[k];
  const int lane = threadIdx.x & 31;
  const int s_m = S.s_m, s_r = S.s_mr;
  const ParamsDev& P = L.prm;
  const int n_sub = L.n_tiles * SPT;
  const int cp = pass & 1;
  const long long gl = (long long)w.z + lane * EPL;   // the lane's first element
  const int nl = w.w - lane * EPL;                    // its members (<= 0: none)
  const V4* wr = (const V4*)L.wr;
  const R m0 = sizeof(R) == 4 ? (R)L.p.m0f : (R)L.p.m0;
  // the lane's elements, all in flight at once
  V4 q[EPL];
  R mq[EPL], uq[EPL];
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const long long g = gl + i;
    if (i < nl) {
      q[i] = wr[g];
      mq[i] = UNIF ? m0 : ((const R*)L.ms)[g];
      uq[i] = GAS ? ((const R*)L.uth)[g] : (R)0;
    } else {
      q[i].x = q[i].y = q[i].z = (R)0;
      q[i].w = neg0(R());
      mq[i] = m0;
      uq[i] = (R)0;
    }
  }
  Acc M, Pp;
  sub_prefix<Acc>(L, u, t, cp, M, Pp, nullptr);
  R vb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) vb[a] = sizeof(R) == 4 ? (R)S.vbulk[a] : (R)S.vbulk_d[a];
  const R band = sizeof(R) == 4 ? (R)P.band_f : (R)P.band;
  const Acc Ttot = Ald<Acc>(S.t_tot);
  const float sc_m = FAST ? pow2_neg(s_m) : 0.0f, sc_r = FAST ? pow2_neg(s_r) : 0.0f;
  const Acc mfix0 = fixp(m0, s_m);
  // per element: 1/r and the exact terms; the lane's sums
  R ri[EPL];
  Acc rf[EPL];
  Acc a = 0, b = 0;
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const bool alive = !signbit(q[i].w);
    ri[i] = rinv_real(q[i].w, P);
    rf[i] = alive ? fixp(mq[i] * ri[i], s_r) : (Acc)0;
    if (alive) a += UNIF ? mfix0 : fixp(mq[i], s_m);
    b += rf[i];
  }
  const Acc ia = wscan(a, lane), ib = wscan(b, lane);
  M += ia - a;
  Pp += ib - b;
  const size_t jc = (size_t)cp * n_sub + u;
  const Acc n_m = ((const Acc*)L.agg_m)[jc], n_r = ((const Acc*)L.agg_r)[jc];
  const int n_c = L.agg_c[jc];
  // phi and the escape test; the skip record's margin and |u| over the
  // members left alive
  unsigned rem = 0;
  int nband = 0;
  Acc rm = 0, rr = 0;
  const R keep_frac = (R)1 - band - (R)0x1p-16;
  R mg = (R)INFINITY, uu = (R)0;
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const R r = q[i].w;
    if (!signbit(r)) {
      const Acc mfix = UNIF ? mfix0 : fixp(mq[i], s_m);
      const R Mf = (FAST && sizeof(R) == 4) ? (R)fix_to_float_sc((long long)M, sc_m) : from_fix(M, s_m, R());
      const R Sf = (FAST && sizeof(R) == 4) ? (R)fix_to_float_sc((long long)(Ttot - Pp), sc_r)
                                            : from_fix(Ttot - Pp, s_r, R());
      const R phi = phi_real(Mf, ri[i], Sf, P);
      const R ux = q[i].x - vb[0], uy = q[i].y - vb[1], uz = q[i].z - vb[2];
      const R uk = fma_x(uz, uz, fma_x(uy, uy, ux * ux));
      R u2 = uk;
      if (GAS) u2 += (R)2 * uq[i];                 // gas: |u|^2 + 2 u_th (Sect. 2.1)
      const R two_phi = (R)-2 * phi;
      if (fabs(u2 - two_phi) < band * two_phi) ++nband;
      if (u2 > two_phi) {
        rem |= 1u << i;
        rm += mfix;
        rr += rf[i];
      } else {
        mg = fmin(mg, two_phi * keep_frac - u2);
        uu = fmax(uu, uk);
      }
      M += mfix;
      Pp += rf[i];
    }
  }
  write_skip<R>(L, u, S, mg, uu, q[0].w, vb);
  // the sub-tile's sums after the removals (next copy) and its removal flags
  const int nrem = __reduce_add_sync(FULL_MASK, __popc(rem));
  nband = __reduce_add_sync(FULL_MASK, nband);
  L.rem_mask[(size_t)u * 32 + lane] = (uint8_t)rem;
  if (nrem) {                                      // uniform over the warp
    rm = wsum(rm);
    rr = wsum(rr);
  }
  if (lane == 0) {
    const size_t j = (size_t)(cp ^ 1) * n_sub + u;
    ((Acc*)L.agg_m)[j] = n_m - rm;
    ((Acc*)L.agg_r)[j] = n_r - rr;
    L.agg_c[j] = n_c - nrem;
    if (nband) atomicAdd((unsigned long long*)&S.band_pass, (unsigned long long)nband);
  }
}

// One pass: warps take the listed sub-tiles (those of the active haloes)
// round robin, and clear the count of the next pass's list.
template <typename R, bool UNIF, bool GAS>
__global__ void __launch_bounds__(T, sizeof(R) == 4 ? 2 : 1) g_pass(GridLaunch L, int pass) {
  if (blockIdx.x == 0 && threadIdx.x == 0) L.ctl->work_n[(pass + 1) & 1] = 0;
  if (gave_up(L)) return;
  const int n = __ldcg(&L.ctl->work_n[pass & 1]);
  const int4* list = L.work + (size_t)(pass & 1) * L.n_tiles * SPT;
  for (int i = (blockIdx.x * T + threadIdx.x) >> 5; i < n; i += (gridDim.x * T) >> 5) {
    const int4 w = list[i];
    const GridHaloState& S = L.state[w.y];
    if (sizeof(R) == 4 && pow2_neg(S.s_m) != 0.0f && pow2_neg(S.s_mr) != 0.0f)
      pass_sub<R, UNIF, GAS, true>(L, w, pass);
    else
      pass_sub<R, UNIF, GAS, false>(L, w, pass);
  }
}

// After a pass, the particles it removed (the flags of the listed sub-tiles):
// the sign bit of r, their removal iteration, and the exact sum m v of what
// each halo lost (v from the candidate's record), one warp per sub-tile.
template <typename R, bool UNIF>
__global__ void __launch_bounds__(T) g_removed(GridLaunch L, int pass) {
  if (gave_up(L)) return;
  using V4 = typename Prec<R>::V4;
  using Acc = typename Prec<R>::Acc;
  const int lane = threadIdx.x & 31;
  const int n = __ldcg(&L.ctl->work_n[pass & 1]);
  const int4* list = L.work + (size_t)(pass & 1) * L.n_tiles * SPT;
  V4* wr = (V4*)L.wr;
  const V4* rec = (const V4*)L.rec;
  const R m0 = sizeof(R) == 4 ? (R)L.p.m0f : (R)L.p.m0;
  // 32 listed sub-tiles per step: lane j checks entry i0 + j's flags (32
  // bytes), then the warp takes the flagged ones one after another
  const int nwarps = (gridDim.x * T) >> 5;
  for (int i0 = ((blockIdx.x * T + threadIdx.x) >> 5) * 32; i0 < n; i0 += nwarps * 32) {
    const int ij = i0 + lane;
    int4 wj = make_int4(0, 0, 0, 0);
    bool any = false;
    if (ij < n) {
      wj = list[ij];
      const uint4* mk = (const uint4*)(L.rem_mask + (size_t)wj.x * 32);
      const uint4 m0 = mk[0], m1 = mk[1];
      any = (m0.x | m0.y | m0.z | m0.w | m1.x | m1.y | m1.z | m1.w) != 0u;
    }
    unsigned todo = __ballot_sync(FULL_MASK, any);
    while (todo) {
    const int jj = __ffs(todo) - 1;
    todo &= todo - 1;
    int4 w;
    w.x = __shfl_sync(FULL_MASK, wj.x, jj);
    w.y = __shfl_sync(FULL_MASK, wj.y, jj);
    w.z = __shfl_sync(FULL_MASK, wj.z, jj);
    w.w = __shfl_sync(FULL_MASK, wj.w, jj);
    unsigned rem = L.rem_mask[(size_t)w.x * 32 + lane];
    GridHaloState& S = L.state[w.y];
    const HaloDev& H = L.halos[w.y];
    const int s_v = S.s_mv;
    Acc mv0 = 0, mv1 = 0, mv2 = 0;
    if (rem) {
      // the lane's removed elements: their candidate positions, then their
      // records, each round's loads issued together
      const long long g0 = (long long)w.z + lane * EPL;
      uint32_t pos[EPL];
#pragma unroll
      for (int e = 0; e < EPL; ++e)
        if ((rem >> e) & 1u) pos[e] = L.val_x[g0 + e];
      V4 vm[EPL];
#pragma unroll
      for (int e = 0; e < EPL; ++e)
        if ((rem >> e) & 1u) vm[e] = rec[2 * (H.gbase + pos[e]) + 1];  // (v, m) of the candidate
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        if (!((rem >> e) & 1u)) continue;
        const long long g = g0 + e;
        // removed: the sign bit of r, set without reading r
        if (sizeof(R) == 4) atomicOr((unsigned*)&wr[g].w, 0x80000000u);
        else atomicOr((unsigned long long*)&wr[g].w, 0x8000000000000000ull);
        if (L.out.removed_iter) L.out.removed_iter[H.offset + pos[e]] = pass;
        const R m = UNIF ? m0 : ((const R*)L.ms)[g];
        mv0 += fixr(mul_rn(m, vm[e].x), s_v);
        mv1 += fixr(mul_rn(m, vm[e].y), s_v);
        mv2 += fixr(mul_rn(m, vm[e].z), s_v);
      }
    }
    mv0 = wsum(mv0);
    mv1 = wsum(mv1);
    mv2 = wsum(mv2);
    if (lane == 0) {
      atomic_acc(S.rem_mv[0], mv0);
      atomic_acc(S.rem_mv[1], mv1);
      atomic_acc(S.rem_mv[2], mv2);
    }
    }
  }
}

// ---- the pass with tensor copies into shared memory (mixed mode) -----------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// One 4 KB box (32 rows of 8 elements) of the stream into dst; bar counts it.
__device__ __forceinline__ void tma_box(void* dst, const CUtensorMap* map, int row, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 4096;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(0), "r"(row), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Wait for a barrier phase with at most `limit` polls; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, long long limit) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_test(bar, phase)) return true;
  return false;
}
constexpr long long DRAIN_POLLS = 1ll << 24;   // a warp that gave up still lets its copies land

// Element i of lane `lane` of a box copied with the 128-byte swizzle: row
// `lane`, 16-byte chunk i stored at chunk i ^ (lane & 7).
__device__ __forceinline__ float4 box_at(const float4* box, int lane, int i) { return box[lane * 8 + (i ^ (lane & 7))]; }

// One sub-tile from its box in shared memory (the mixed mode, a uniform
// particle mass, no gas): the arithmetic of pass_sub.
template <bool FAST>
__device__ __forceinline__ void pass_box(const GridLaunch& L, const int4 w, int pass, const float4* box) {
  using Acc = long long;
  const int u = w.x, k = w.y, t = u / SPT;
  GridHaloState& S = L.state[k];
  const int lane = threadIdx.x & 31;
  const int s_m = S.s_m, s_r = S.s_mr;
  const ParamsDev& P = L.prm;
  const int n_sub = L.n_tiles * SPT;
  const int cp = pass & 1;
  const int nl = w.w - lane * EPL;                    // the lane's members (<= 0: none)
  Acc M, Pp;
  sub_prefix<Acc>(L, u, t, cp, M, Pp, nullptr);
  const float vb0 = S.vbulk[0], vb1 = S.vbulk[1], vb2 = S.vbulk[2];
  const float band = P.band_f;
  const Acc Ttot = Ald<Acc>(S.t_tot);
  const float sc_m = FAST ? pow2_neg(s_m) : 0.0f, sc_r = FAST ? pow2_neg(s_r) : 0.0f;
  const float m0 = L.p.m0f;
  const Acc mfix0 = fixp(m0, s_m);
  float ri[EPL];
  Acc rf[EPL];
  Acc a = 0, b = 0;
  unsigned alive = 0;
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const float r = box_at(box, lane, i).w;
    const bool al = i < nl && !signbit(r);
    alive |= (al ? 1u : 0u) << i;
    ri[i] = rinv_real(r, P);
    rf[i] = al ? fixp(m0 * ri[i], s_r) : 0ll;
    a += al ? mfix0 : 0ll;
    b += rf[i];
  }
  const Acc ia = wscan(a, lane), ib = wscan(b, lane);
  M += ia - a;
  Pp += ib - b;
  const size_t jc = (size_t)cp * n_sub + u;
  const Acc n_m = ((const Acc*)L.agg_m)[jc], n_r = ((const Acc*)L.agg_r)[jc];
  const int n_c = L.agg_c[jc];
  unsigned rem = 0;
  int nband = 0;
  Acc rr = 0;
  const float keep_frac = 1.0f - band - 0x1p-16f;
  float mg = INFINITY, uu = 0.0f;
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    if (alive & (1u << i)) {
      const float4 q = box_at(box, lane, i);
      const float Mf = FAST ? fix_to_float_sc(M, sc_m) : float_from_fix(M, s_m);
      const float Sf = FAST ? fix_to_float_sc(Ttot - Pp, sc_r) : float_from_fix(Ttot - Pp, s_r);
      const float phi = phi_of(Mf, ri[i], Sf, P.Gf);
      const float ux = q.x - vb0, uy = q.y - vb1, uz = q.z - vb2;
      const float u2 = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
      const float two_phi = -2.0f * phi;
      if (fabsf(u2 - two_phi) < band * two_phi) ++nband;
      if (u2 > two_phi) {
        rem |= 1u << i;
        rr += rf[i];
      } else {
        mg = fminf(mg, fmaf(two_phi, keep_frac, -u2));
        uu = fmaxf(uu, u2);
      }
      M += mfix0;
      Pp += rf[i];
    }
  }
  {
    const float vbv[3] = {vb0, vb1, vb2};
    write_skip<float>(L, u, S, mg, uu, box_at(box, lane, 0).w, vbv);
  }
  const int nrem = __reduce_add_sync(FULL_MASK, __popc(rem));
  nband = __reduce_add_sync(FULL_MASK, nband);
  L.rem_mask[(size_t)u * 32 + lane] = (uint8_t)rem;
  if (nrem) rr = wsum(rr);
  if (lane == 0) {
    const size_t j = (size_t)(cp ^ 1) * n_sub + u;
    ((Acc*)L.agg_m)[j] = n_m - (Acc)nrem * mfix0;
    ((Acc*)L.agg_r)[j] = n_r - rr;
    L.agg_c[j] = n_c - nrem;
    if (nband) atomicAdd((unsigned long long*)&S.band_pass, (unsigned long long)nband);
  }
}

// One pass with the sub-tiles streamed into shared memory by tensor copies:
// each warp keeps two 4 KB boxes, fetching its next sub-tile while it
// computes the current one.  Waits are bounded by L.wait_limit polls; a warp
// that gives up sets ERR_TIMEOUT, lets its copies land and stops.
constexpr int TMA_SMEM = NWARP * 2 * 4096 + NWARP * 2 * 8;
__global__ void __launch_bounds__(T, 3) g_pass_tma(const __grid_constant__ GridLaunch L, int pass) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* box0 = (float4*)(smem + warp * 8192);
  uint64_t* bar = (uint64_t*)(smem + NWARP * 8192) + 2 * warp;
  if (blockIdx.x == 0 && threadIdx.x == 0) L.ctl->work_n[(pass + 1) & 1] = 0;
  if (gave_up(L)) return;
  const int n = __ldcg(&L.ctl->work_n[pass & 1]);
  const int4* list = L.work + (size_t)(pass & 1) * L.n_tiles * SPT;
  const int stride = gridDim.x * NWARP;
  int i = blockIdx.x * NWARP + warp;
  if (i >= n) return;
  if (smem_u32(smem) & 1023) {                       // the swizzled boxes need 1 KB alignment
    if (lane == 0) atomicOr(L.out.err, ERR_TIMEOUT);
    return;
  }
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_async_smem();
  }
  __syncwarp();
  uint32_t phase0 = 0, phase1 = 0;
  int4 w = list[i];
  if (lane == 0) tma_box(box0, &L.wr_map, w.z >> 3, &bar[0]);
  for (int b = 0; i < n; i += stride, b ^= 1) {
    const int inext = i + stride;
    const int4 wn = inext < n ? list[inext] : make_int4(0, 0, 0, 0);
    __syncwarp();
    if (inext < n && lane == 0) {
      fence_async_smem();
      tma_box(box0 + (b ^ 1) * 256, &L.wr_map, wn.z >> 3, &bar[b ^ 1]);
    }
    const uint32_t ph = b ? phase1 : phase0;
    if (!mbar_wait(&bar[b], ph, L.wait_limit)) {
      if (lane == 0) atomicOr(L.out.err, ERR_TIMEOUT);
      mbar_wait(&bar[b], ph, DRAIN_POLLS);
      if (inext < n) mbar_wait(&bar[b ^ 1], b ? phase0 : phase1, DRAIN_POLLS);
      return;
    }
    if (b) phase1 ^= 1;
    else phase0 ^= 1;
    const GridHaloState& S = L.state[w.y];
    if (pow2_neg(S.s_m) != 0.0f && pow2_neg(S.s_mr) != 0.0f) pass_box<true>(L, w, pass, box0 + b * 256);
    else pass_box<false>(L, w, pass, box0 + b * 256);
    w = wn;
  }
}

// ---- final pass --------------------------------------------------------------------------

// Bound lists (radial order), phi of the final set, compacted radius and
// inclusive mass for the virial search and the profile rows; one warp per
// sub-tile, lanes holding consecutive elements as in a pass.
template <typename R, bool UNIF>
__global__ void __launch_bounds__(T, sizeof(R) == 4 ? 4 : 2) g_final(GridLaunch L) {
  if (gave_up(L)) return;
  using V4 = typename Prec<R>::V4;
  using Acc = typename Prec<R>::Acc;
  const int lane = threadIdx.x & 31;
  const int n_sub = L.n_tiles * SPT;
  const int u = (blockIdx.x * T + threadIdx.x) >> 5;     // one warp per sub-tile
  if (u >= n_sub) return;
  const V4* wr = (const V4*)L.wr;
  R* rc = (R*)L.rc;
  Acc* mc = (Acc*)L.mc;
  const R m0 = sizeof(R) == 4 ? (R)L.p.m0f : (R)L.p.m0;
  const ParamsDev& P = L.prm;
  const int t = u / SPT;
  const int2 tr = L.tile_range[t];
  const int e0 = (u % SPT) * SUB;
  // rows of 32 consecutive elements (coalesced), read before the halo's
  // state arrives; elements past the last member count as removed
  R rq[ROWS], mq[ROWS];
  uint32_t vq[ROWS];
#pragma unroll
  for (int i = 0; i < ROWS; ++i) {
    const int e = e0 + 32 * i + lane;
    const long long g = (long long)tr.x + e;
    rq[i] = e < tr.y ? wr[g].w : neg0(R());
    mq[i] = (!UNIF && e < tr.y) ? ((const R*)L.ms)[g] : m0;
    vq[i] = e < tr.y ? L.val_x[g] : 0u;
  }
  const int k = L.tile_halo[t];
  const GridHaloState& S = L.state[k];
  if (S.n_alive == 0) return;
  const HaloDev& H = L.halos[k];
  const long long lim = H.gbase + S.n_member;
  const int s_m = S.s_m, s_r = S.s_mr;
  const Acc Ttot = Ald<Acc>(S.t_tot);
  Acc M, Pp;
  long long C;
  sub_prefix<Acc>(L, u, t, (S.n_iter + 1) & 1, M, Pp, &C);
  const float sc_m = pow2_neg(s_m), sc_r = pow2_neg(s_r);
  const unsigned below = lanemask_lt();
#pragma unroll
  for (int i = 0; i < ROWS; ++i) {
    const R r = rq[i];
    const bool alive = !signbit(r) && (long long)tr.x + e0 + 32 * i + lane < lim;
    const R ri = rinv_real(r, P);
    const Acc a = alive ? (Acc)fixp(mq[i], s_m) : (Acc)0;
    const Acc b = alive ? (Acc)fixp(mq[i] * ri, s_r) : (Acc)0;
    const unsigned bal = __ballot_sync(FULL_MASK, alive);
    if (bal == 0u) continue;
    const Acc ia = wscan(a, lane), ib = wscan(b, lane);
    if (alive) {
      // M(<r) before the particle, and the outer sum from the particle out
      const R phi = phi_real(fix_to_real(M + ia - a, s_m, sc_m, R()), ri,
                             fix_to_real(Ttot - (Pp + ib - b), s_r, sc_r, R()), P);
      const long long slot = H.offset + vq[i];
      const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
      const long long c = C + __popc(bal & below);
      L.out.bound_idx[H.offset + c] = pi;
      if (L.out.phi) ((R*)L.out.phi)[H.offset + c] = phi;
      rc[H.gbase + c] = r;
      mc[H.gbase + c] = M + ia;
    }
    M += shfl_idx_x(ia, 31);
    Pp += shfl_idx_x(ib, 31);
    C += __popc(bal);
  }
}

// First compacted index k with M_k < delta_rho 4pi/3 r_{k+1}^3 (r_{N+1} = inf).
template <typename R>
__global__ void __launch_bounds__(T) g_virial(GridLaunch L) {
  if (gave_up(L)) return;
  using Acc = typename Prec<R>::Acc;
  const R* rc = (const R*)L.rc;
  const Acc* mc = (const Acc*)L.mc;
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
      const Acc mk = mc[g];
      if (sizeof(R) == 4) {
        const float rn = (float)rc[g + 1];
        const float lhs = from_fix(mk, S.s_m, R());
        const float rhs = P.crit_f * rn * rn * rn;
        if (lhs < rhs * (1.0f - 1e-5f)) cross = true;
        else if (lhs > rhs * (1.0f + 1e-5f)) cross = false;
        else {
          const double rd = (double)rn;
          cross = dfix(mk, S.s_m) < P.crit * rd * rd * rd;
        }
      } else {
        const double rd = (double)rc[g + 1];
        const double mkd = L.p.m == nullptr ? (double)(kk + 1) * L.p.m0 : dfix(mk, S.s_m);
        cross = mkd < P.crit * rd * rd * rd;
      }
    }
    if (cross) {
      kf = kk;
      break;
    }
  }
  for (int o = 16; o > 0; o >>= 1) kf = min(kf, __shfl_xor_sync(FULL_MASK, kf, o));
  if ((threadIdx.x & 31) == 0 && kf != 0x7fffffffffffffffll)
    atomicMin((unsigned long long*)&S.k_first, (unsigned long long)kf);
}

template <typename R>
__global__ void g_result(GridLaunch L) {
  if (gave_up(L)) return;
  using Acc = typename Prec<R>::Acc;
  const R* rc = (const R*)L.rc;
  const Acc* mcv = (const Acc*)L.mc;
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
    const Acc mkx = unim ? (Acc)0 : mcv[H.gbase + kk];
    const double mk = unim ? double_from_fix(kk + 1, 0) * L.p.m0 : dfix(mkx, S.s_m);
    if (kk == nb - 1) status |= AHF_HALO_RVIR_BEYOND_EDGE;
    bool none;
    if (sizeof(R) == 4) {
      // the decision and the values as in the on-chip classes (the same bits)
      const float mkf = unim ? (float)(kk + 1) * L.p.m0f : (float)from_fix(mkx, S.s_m, R());
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
        auto at = [&](long long j, double& r, double& m) {
          r = sizeof(R) == 4 ? float_to_double((float)rc[H.gbase + j]) : (double)rc[H.gbase + j];
          m = unim ? double_from_fix(j + 1, 0) * L.p.m0 : dfix(mcv[H.gbase + j], S.s_m);
        };
        const long long ke = rise_edge_index(nb, at);
        if (ke >= 0) {
          at(ke, Rs.r_vir, Rs.m_vir);
          Rs.k_vir = ke;
          status |= AHF_HALO_RISE_EDGE;
        }
      }
    }
    const double mt = dfix(Ald<Acc>(S.m_tot), S.s_m);
    for (int a = 0; a < 3; ++a) Rs.vbulk[a] = quotient(dfix(Ald<Acc>(S.mv[a]), S.s_mv), mt);
  } else {
    Rs.vbulk[0] = Rs.vbulk[1] = Rs.vbulk[2] = 0.0;
  }
  Rs.status = status;
  L.out.res[H.index] = Rs;
}

// Profile rows of every halo of the class from its compacted bound set (one
// CTA per halo, the rows spread over the threads; Sect. 2.1's radially binned
// output): each edge by binary search over the compacted radii.
__global__ void __launch_bounds__(T) g_rows_mixed(GridLaunch L) {
  if (gave_up(L)) return;
  const int k = blockIdx.x;
  const HaloDev& H = L.halos[k];
  const GridHaloState& S = L.state[k];
  const ahf_result& Rs = L.out.res[H.index];
  const double m0 = L.p.m0;
  const long long gb = H.gbase;
  profile_rows(L.rows, H.index, (const float*)L.rc, (const long long*)L.mc, [gb](long long j) { return gb + j; },
               S.n_alive, Rs.r_vir, S.s_m, L.prm.G, L.prm.Gf, L.p.m == nullptr ? &m0 : nullptr, threadIdx.x, T);
}

// The all-FP64 rows: FP64 radii against the FP64 edges, __int128 masses.
__global__ void __launch_bounds__(T) g_rows_f64(GridLaunch L) {
  if (gave_up(L)) return;
  const int k = blockIdx.x;
  const HaloDev& H = L.halos[k];
  const GridHaloState& S = L.state[k];
  const ahf_result& Rs = L.out.res[H.index];
  const ProfileRows& Q = L.rows;
  const int n = Q.n_bins;
  double* out = Q.prof + (size_t)H.index * n * 4;
  const long long nb = S.n_alive;
  const double* rc = (const double*)L.rc + H.gbase;
  const __int128* mc = (const __int128*)L.mc + H.gbase;
  if (nb == 0) {
    for (int i = threadIdx.x; i < 4 * n; i += T) out[i] = 0.0;
    return;
  }
  const double r_out = Rs.r_vir > 0.0 ? Rs.r_vir : rc[nb - 1];
  const float inv_r = 1.0f / double_to_float(r_out);
  auto count_le = [&](int b) {               // first j with rc[j] > e_b (b = n: r_out)
    const double e = b == n ? r_out : r_out * Q.factor[b];
    long long lo = 0, hi = nb;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (rc[mid] <= e) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  for (int b = threadIdx.x; b < n; b += T) {
    const long long c0 = count_le(b), c1 = count_le(b + 1);
    double M1, Mshell;
    if (L.p.m == nullptr) {
      M1 = double_from_fix(c1, 0) * L.p.m0;
      Mshell = double_from_fix(c1 - c0, 0) * L.p.m0;
    } else {
      const __int128 f0 = c0 > 0 ? mc[c0 - 1] : (__int128)0;
      const __int128 f1 = c1 > 0 ? mc[c1 - 1] : (__int128)0;
      M1 = double_from_fix128(f1, S.s_m);
      Mshell = double_from_fix128(f1 - f0, S.s_m);
    }
    out[4 * b + 0] = double_from_fix(c1 - c0, 0);
    out[4 * b + 1] = M1;
    out[4 * b + 2] = shell_density(Mshell, r_out, inv_r, Q.factor, Q.factor_f, n, b);
    out[4 * b + 3] = circular_velocity(L.prm.G, L.prm.Gf, M1, r_out, inv_r, Q.factor, Q.factor_f, n, b);
  }
}

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

template <typename R>
cudaError_t prepare_t(const GridLaunch& L, cudaStream_t s) {
  if (L.n_tiles == 0) {
  } else if (sizeof(R) == 4) {
    if (L.p.coord_type == AHF_COORD_F64) g_prepare_mixed<AHF_COORD_F64><<<L.n_tiles, T, 0, s>>>(L);
    else g_prepare_mixed<AHF_COORD_F32_REL><<<L.n_tiles, T, 0, s>>>(L);
  } else {
    if (L.p.coord_type == AHF_COORD_F64) g_prepare_f64<AHF_COORD_F64><<<L.n_tiles, T, 0, s>>>(L);
    else g_prepare_f64<AHF_COORD_F32_REL><<<L.n_tiles, T, 0, s>>>(L);
  }
  g_scales<R><<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

template <typename R>
cudaError_t sort_t(GridLaunch& L, cudaStream_t s, unsigned long long or_bits, unsigned long long and_bits) {
  using Key = typename Prec<R>::Key;
  const unsigned long long diff = or_bits ^ and_bits;
  int digits[8];
  int nd = 0;
  for (int d = 0; d < (int)sizeof(Key); ++d)
    if ((diff >> (8 * d)) & 0xffull) digits[nd++] = d;
  if (L.n_tiles == 0) nd = 0;
  L.sort_passes = nd;
  L.sort_launches = 0;
  if (L.n_tiles == 0) return cudaGetLastError();
  Key *ki = (Key*)L.key_a, *ko = (Key*)L.key_b;
  uint32_t *vi = L.val_a, *vo = L.val_b;
  for (int p = 0; p < nd; ++p) {
    const int shift = 8 * digits[p];
    // the prepare left the low byte's tile counts
    if (p > 0 || shift != 0) {
      g_hist<Key><<<L.n_tiles, T, 0, s>>>(ki, L.tile_range, L.tile_halo, L.halo_tile0, L.tile_hist, shift);
      ++L.sort_launches;
    }
    L.sort_launches += 3 + (L.n_big ? 1 : 0);
    g_digit_scan_small<<<L.n_halos, 256, 0, s>>>(L.tile_hist, L.halo_tile0, L.digit_base);
    if (L.n_big) g_digit_scan_big<<<L.n_big * 256, 256, 0, s>>>(L.tile_hist, L.halo_tile0, L.big_halos, L.digit_base);
    g_digit_base<<<L.n_halos, 256, 0, s>>>(L.digit_base);
    const bool first = p == 0, last = p == nd - 1;
    if (first && last) g_scatter<Key, R, true, true><<<L.n_tiles, T, 0, s>>>(L, ki, vi, ko, vo, shift);
    else if (first) g_scatter<Key, R, true, false><<<L.n_tiles, T, 0, s>>>(L, ki, vi, ko, vo, shift);
    else if (last) g_scatter<Key, R, false, true><<<L.n_tiles, T, 0, s>>>(L, ki, vi, ko, vo, shift);
    else g_scatter<Key, R, false, false><<<L.n_tiles, T, 0, s>>>(L, ki, vi, ko, vo, shift);
    Key* x = ki;
    ki = ko;
    ko = x;
    uint32_t* y = vi;
    vi = vo;
    vo = y;
  }
  if (nd == 0) g_fill_identity<R><<<L.n_tiles, T, 0, s>>>(L);
  L.sort_launches += (nd == 0 ? 1 : 0) + 2;
  g_sums<R><<<(int)(((long long)L.n_tiles * SPT + NWARP - 1) / NWARP), T, 0, s>>>(L);
  if (L.max_halo_tiles > 64) g_halo<R, true, HT_BIG><<<L.n_halos, HT_BIG, 0, s>>>(L, 0);
  else g_halo<R, true, HT_SMALL><<<L.n_halos, HT_SMALL, 0, s>>>(L, 0);
  return cudaGetLastError();
}

std::atomic<unsigned long long> g_tma_attr{0};

template <typename R>
cudaError_t iterate_t(const GridLaunch& L, int pass, cudaStream_t s) {
  const bool unif = L.ms == nullptr, gas = L.uth != nullptr;
  if (sizeof(R) == 4 && L.use_tma && unif && !gas) {
    if (first_use_on_device(g_tma_attr)) {
      const cudaError_t e = cudaFuncSetAttribute(g_pass_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM);
      if (e != cudaSuccess) return e;
      mark_used_on_device(g_tma_attr);
    }
    g_pass_tma<<<L.tma_grid, T, TMA_SMEM, s>>>(L, pass);
  } else if (unif && !gas) g_pass<R, true, false><<<L.iter_grid, T, 0, s>>>(L, pass);
  else if (!unif && !gas) g_pass<R, false, false><<<L.iter_grid, T, 0, s>>>(L, pass);
  else if (unif) g_pass<R, true, true><<<L.iter_grid, T, 0, s>>>(L, pass);
  else g_pass<R, false, true><<<L.iter_grid, T, 0, s>>>(L, pass);
  if (unif) g_removed<R, true><<<L.iter_grid, T, 0, s>>>(L, pass);
  else g_removed<R, false><<<L.iter_grid, T, 0, s>>>(L, pass);
  if (L.max_halo_tiles > 64) g_halo<R, false, HT_BIG><<<L.n_halos, HT_BIG, 0, s>>>(L, pass);
  else g_halo<R, false, HT_SMALL><<<L.n_halos, HT_SMALL, 0, s>>>(L, pass);
  return cudaGetLastError();
}

template <typename R>
cudaError_t finish_t(const GridLaunch& L, cudaStream_t s) {
  if (L.n_tiles > 0) {
    const int nb = (int)(((long long)L.n_tiles * SPT + NWARP - 1) / NWARP);
    if (L.ms == nullptr) g_final<R, true><<<nb, T, 0, s>>>(L);
    else g_final<R, false><<<nb, T, 0, s>>>(L);
    g_virial<R><<<L.n_tiles, T, 0, s>>>(L);
  }
  g_result<R><<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  if (L.rows.prof) {
    if (sizeof(R) == 4) g_rows_mixed<<<L.n_halos, T, 0, s>>>(L);
    else g_rows_f64<<<L.n_halos, T, 0, s>>>(L);
  }
  return cudaGetLastError();
}

template <typename R>
int iter_grid_t(int device) {
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, g_pass<R, true, false>, T, 0) != cudaSuccess) return 0;
  return sms * (per > 0 ? per : 1);
}

}  // namespace

int grid_iter_grid(int device, int fp64) { return fp64 ? iter_grid_t<double>(device) : iter_grid_t<float>(device); }

int grid_tma_grid(int device) {
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(g_pass_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, g_pass_tma, T, TMA_SMEM) != cudaSuccess) return 0;
  return sms * per;
}

// The stream (w, r) of n_rows 8-element rows as a 2-D float tensor of 32
// columns, copied in boxes of 32 x 32 (4 KB) with the 128-byte swizzle.
bool grid_wr_map(GridLaunch& L, long long n_rows) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = (Encode)fn;
    cudaGetLastError();
  }
  if (!encode || n_rows <= 0 || ((uintptr_t)L.wr & 15)) return false;
  const cuuint64_t dims[2] = {32, (cuuint64_t)n_rows};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  return encode(&L.wr_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, L.wr, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t grid_prepare(const GridLaunch& L, cudaStream_t s) {
  return L.fp64 ? prepare_t<double>(L, s) : prepare_t<float>(L, s);
}

cudaError_t grid_sort(GridLaunch& L, cudaStream_t s, unsigned long long or_bits, unsigned long long and_bits) {
  return L.fp64 ? sort_t<double>(L, s, or_bits, and_bits) : sort_t<float>(L, s, or_bits, and_bits);
}

cudaError_t grid_iterate(const GridLaunch& L, int pass, cudaStream_t s) {
  return L.fp64 ? iterate_t<double>(L, pass, s) : iterate_t<float>(L, pass, s);
}

cudaError_t grid_finish(const GridLaunch& L, cudaStream_t s) {
  return L.fp64 ? finish_t<double>(L, s) : finish_t<float>(L, s);
}

}  // namespace ahf
