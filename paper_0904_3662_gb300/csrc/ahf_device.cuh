// Device-side building blocks shared by the libahfgpu kernels.
//
// Exact sums.  GB300 runs FP64 adds at about 1/70 of the FP32 rate, so the
// sums the method needs beyond FP32 precision -- M(<r), sum m/r, sum m v and
// sum m (Appendix A, Sect. 2.1) -- are accumulated in 64-bit fixed point on
// the integer pipes.  A halo-wide scale 2^s is picked from the largest term's
// exponent and the member count so that no partial sum can overflow; each
// term is rounded once when it is converted, after which every addition is
// exact.  The result therefore does not depend on the order of the additions
// (tile size, CTA count, batch composition), which a tree of FP64 adds cannot
// promise.
#pragma once

#include <atomic>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "ahf_internal.h"

namespace ahf {

// True the first time it is called for this kernel (its `mask`) on the
// current device: function attributes persist for the process, so they are
// set once rather than on every launch.
inline bool first_use_on_device(std::atomic<unsigned long long>& mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
  const unsigned long long bit = 1ull << dev;
  return (mask.load(std::memory_order_acquire) & bit) == 0;
}
inline void mark_used_on_device(std::atomic<unsigned long long>& mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) mask.fetch_or(1ull << dev, std::memory_order_release);
}

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr uint32_t KEY_NONMEMBER = 0xffffffffu;   // sorts after every r >= 0

// ---- fixed point ------------------------------------------------------------

// Scale exponent s for sums of n terms of magnitude < 2^(emax+1): every
// partial sum of term * 2^s stays below 2^62.
__host__ __device__ __forceinline__ int fix_scale(int emax, long long n) {
  int bits = 0;
  while (bits < 40 && (1ll << bits) < n) ++bits;
  return 61 - bits - emax;
}

// Unbiased exponent of a positive finite float (floor(log2 x)); -127 for 0.
__device__ __forceinline__ int float_exponent_of_bits(uint32_t bits) {
  return (int)((bits >> 23) & 0xff) - 127;
}

// round(x * 2^s) in integer arithmetic (round half away from zero).  The
// caller guarantees |x| * 2^s < 2^62.
__device__ __forceinline__ long long fix_from_float(float x, int s) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xff);
  if (e == 0) return 0;                                   // zero / subnormal
  const long long mant = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 150 + s;
  long long v;
  if (sh >= 0) v = mant << (sh > 39 ? 39 : sh);
  else if (sh > -25) v = ((mant >> (-sh - 1)) + 1) >> 1;
  else v = 0;
  return (b >> 31) ? -v : v;
}

__device__ __forceinline__ long long fix_from_double(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0;
  const long long mant = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = e - 1075 + s;
  long long v;
  if (sh >= 0) v = mant << (sh > 10 ? 10 : sh);
  else if (sh > -54) v = ((mant >> (-sh - 1)) + 1) >> 1;
  else v = 0;
  return (b >> 63) ? -v : v;
}

// f * 2^e for any e (two steps when 2^e is outside the normal float range).
__device__ __forceinline__ float scale_pow2f(float f, int e) {
  while (e > 126) { f *= 8.5070592e37f; e -= 126; }          // 2^126
  while (e < -126) { f *= 1.1754944e-38f; e += 126; }        // 2^-126
  return f * __int_as_float((e + 127) << 23);
}

__host__ __device__ __forceinline__ double scale_pow2d(double f, int e) {
  while (e > 1000) { f *= 1.0715086071862673e301; e -= 1000; }   // 2^1000
  while (e < -1000) { f *= 9.332636185032189e-302; e += 1000; }  // 2^-1000
  // 2^e as a double built from its exponent bits
  union { unsigned long long u; double d; } p;
  p.u = (unsigned long long)(e + 1023) << 52;
  return f * p.d;
}

// int64 -> float using two 32-bit conversions (the 64-bit conversion runs on
// the slow FP64 path on this part), then * 2^-s.  Error within 1 ulp.
__device__ __forceinline__ float float_from_fix(long long v, int s) {
  const float hi = (float)(int)(v >> 32);
  const float lo = (float)(unsigned)(v & 0xffffffffll);
  return scale_pow2f(fmaf(hi, 4294967296.0f, lo), -s);
}

// float_from_fix when 2^-s is the normal float sc (no other route compiled in):
// scale_pow2f multiplies by that same power of two.
__device__ __forceinline__ float fix_to_float_sc(long long v, float sc) {
  const float hi = (float)(int)(v >> 32);
  const float lo = (float)(unsigned)(v & 0xffffffffll);
  return fmaf(hi, 4294967296.0f, lo) * sc;
}
// 2^-s as a float when it is normal, else 0.
__device__ __forceinline__ float pow2_neg(int s) {
  return (s >= -127 && s <= 126) ? __int_as_float((127 - s) << 23) : 0.0f;
}
// float_from_fix(v, s) with sc = pow2_neg(s) computed once per halo.
__device__ __forceinline__ float fix_to_float_fast(long long v, int s, float sc) {
  return sc != 0.0f ? fix_to_float_sc(v, sc) : float_from_fix(v, s);
}

// v 2^-s as the nearest double (ties to even), assembled from the bits on the
// integer pipes: the FP64 pipe of this part is narrow and its latency long, and
// the per-halo record and profile rows would otherwise wait on it.  Results
// outside the normal range take the FP64 route (the same value).
__device__ __forceinline__ double double_from_fix(long long v, int s) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  int e = 63 - __clzll((long long)a);                   // leading bit
  unsigned long long m;
  if (e <= 52) {
    m = a << (52 - e);
  } else {
    const int sh = e - 52;
    m = a >> sh;
    const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m == (1ull << 53)) {
        m >>= 1;
        ++e;
      }
    }
  }
  const int ex = e - s + 1023;
  if (ex <= 0 || ex >= 2047) {
    const double hi = (double)(int)(v >> 32);
    const double lo = (double)(unsigned)(v & 0xffffffffll);
    return scale_pow2d(fma(hi, 4294967296.0, lo), -s);
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) | (m & ((1ull << 52) - 1ull))));
}

// A float as a double (exact), from the bits.
__device__ __forceinline__ double float_to_double(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (double)f;           // zero, subnormal, inf, nan
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)(e - 127u + 1023u) << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// A double rounded to the nearest float (ties to even), from the bits.
__device__ __forceinline__ float double_to_float(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ffull) - 1023 + 127;
  if (e <= 0 || e >= 254) return (float)x;               // outside float's normal range
  uint32_t m = (uint32_t)((u >> 29) & 0x7fffffull);
  const unsigned long long rem = u & ((1ull << 29) - 1ull), half = 1ull << 28;
  uint32_t b = ((uint32_t)e << 23) | m;
  if (rem > half || (rem == half && (m & 1u))) ++b;       // a carry into the exponent is right
  return __uint_as_float(b | (uint32_t)((u >> 63) << 31));
}

// ---- the record's FP64 values from float estimates ---------------------------------

// a / b: q = a r with r the float reciprocal of b, corrected once by the
// residual a - q b in FP64 (the error squares: ~1e-14).
__device__ __forceinline__ double quotient(double a, double b) {
  const float bf = double_to_float(b);
  if (!(fabsf(bf) > 1e-30f && fabsf(bf) < 1e30f)) return a / b;
  const double r = float_to_double(__frcp_rn(bf));
  const double q = a * r;
  return fma(fma(-q, b, a), r, q);
}

// R_vir = (M / crit)^(1/3) with crit = Delta rho_ref 4 pi / 3 (Eq. 1): x = M / crit
// as M inv_crit, a float estimate z of x^(-1/3) and two Newton steps in FP64,
// z <- z + z (1 - x z^3) / 3 (each squares the error: 1e-7 -> 1e-14 -> below
// the FP64 rounding), then x z^2.
__device__ __forceinline__ double virial_radius(double m, double inv_crit) {
  const double x = m * inv_crit;
  const float xf = double_to_float(x);
  if (!(xf > 1e-30f && xf < 1e30f)) return cbrt(x);
  double z = float_to_double(__frcp_rn(cbrtf(xf)));
  z = fma(z * fma(-x, z * z * z, 1.0), 1.0 / 3.0, z);
  z = fma(z * fma(-x, z * z * z, 1.0), 1.0 / 3.0, z);
  return x * (z * z);
}

// Edge of a halo whose mean overdensity never drops below the threshold: the
// rise of its density profile (Sect. 2.1, the truncation of subhaloes).  The
// n bound particles, in radial order, form 16 shells of equal count (shell s
// ends with particle (s+1) n / 16 - 1); among the outer 8 shells the first of
// least density (shell mass over the volume between the radii of the last
// particles of the shell and of the one before, in FP64) is the edge when a
// denser shell lies beyond it.  at(k, r, m) gives particle k's radius and the
// mass up to and including it.  Returns the edge particle's index, or -1.
constexpr int RISE_SHELLS = 16;
constexpr int RISE_MIN_N = 64;
template <typename At>
__device__ long long rise_edge_index(long long n, At at) {
  if (n < RISE_MIN_N) return -1;
  double r_lo, m_lo;
  at((RISE_SHELLS / 2) * n / RISE_SHELLS - 1, r_lo, m_lo);
  double rho_min = 0.0;
  long long k_min = -1;
  bool rise = false;
  for (int s = RISE_SHELLS / 2; s < RISE_SHELLS; ++s) {
    const long long hi = (long long)(s + 1) * n / RISE_SHELLS - 1;
    double r_hi, m_hi;
    at(hi, r_hi, m_hi);
    const double vol = (4.0 * M_PI / 3.0) * (r_hi * r_hi * r_hi - r_lo * r_lo * r_lo);
    const double rho = vol > 0.0 ? (m_hi - m_lo) / vol : INFINITY;
    if (k_min < 0 || rho < rho_min) {
      rho_min = rho;
      k_min = hi;
      rise = false;
    } else if (rho > rho_min) {
      rise = true;
    }
    r_lo = r_hi;
    m_lo = m_hi;
  }
  return rise ? k_min : -1;
}

// m < crit r^3 (the mean density inside r above the threshold fails), in float
// (mf: m rounded) except within 1e-5 of equality, where it is decided in FP64.
__device__ __forceinline__ bool below_threshold(double m, float mf, float r, float crit_f, double crit) {
  const float rhs = crit_f * r * r * r;
  if (mf < rhs * (1.0f - 1e-5f)) return true;
  if (mf > rhs * (1.0f + 1e-5f)) return false;
  const double rd = float_to_double(r);
  return m < crit * rd * rd * rd;
}

// ---- recentring (Sect. 2.1: the sphere around the candidate centre) -----------

// Coordinates are moved to 64-bit fixed point with `frac` fractional bits
// (a float or double below 2^(62-frac) in magnitude converts exactly up to
// bits finer than 2^-frac; anything larger saturates far outside the
// halo), the centre is subtracted as an integer, the result wrapped to the
// minimum image and rounded once to float.  This is the FP64-accurate
// recentring of large box coordinates without FP64 adds.
__device__ __forceinline__ long long fixcoord_from_float(float x, int frac) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xff);
  if (e == 0) return 0;
  const long long mant = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 150 + frac;
  long long v;
  if (sh > 38) v = 1ll << 62;            // far outside every frame: saturate
  else if (sh >= 0) v = mant << sh;
  else if (sh > -25) v = mant >> (-sh);
  else v = 0;
  return (b >> 31) ? -v : v;
}

__device__ __forceinline__ long long fixcoord_from_double(double x, int frac) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0;
  const long long mant = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = e - 1075 + frac;
  long long v;
  if (sh > 8) v = 1ll << 62;             // far outside every frame: saturate
  else if (sh >= 0) v = mant << sh;
  else if (sh > -54) v = mant >> (-sh);
  else v = 0;
  return (b >> 63) ? -v : v;
}

__device__ __forceinline__ long long wrap_fix(long long d, long long box) {
  if (box > 0) {
    const long long half = box >> 1;
    if (d > half) d -= box;
    else if (d < -half) d += box;
  }
  return d;
}

// Round an int64 to the nearest float (ties to even) without the 64-bit
// conversion (which runs on the narrow FP64 pipe of this part): below 2^32 one
// 32-bit conversion; above, the top 32 bits (msb at bit 31, so 8 bits below
// the float's last place) with every bit shifted out ORed into bit 0 (sticky),
// so that the one rounding of the 32-bit conversion sees the whole value, then
// an exact scaling by 2^sh.
__device__ __forceinline__ float f32_from_i64_rn(long long v) {
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const uint32_t hi = (uint32_t)(a >> 32);
  float f;
  if (hi == 0u) {
    f = __uint2float_rn((uint32_t)a);
  } else {
    const int sh = 32 - __clz(hi);                        // 1 .. 32
    uint32_t top = (uint32_t)(a >> sh);
    if (a & ((1ull << sh) - 1ull)) top |= 1u;
    f = __uint2float_rn(top) * __int_as_float((sh + 127) << 23);
  }
  return v < 0 ? -f : f;
}

// Fixed-point offset of one candidate from the halo centre (per axis).
template <int CT>
__device__ __forceinline__ void load_offset_fix(const ParticlesDev& p, long long i, const long long cfix[3],
                                                long long boxfix, int frac, long long f[3]) {
  if (CT == AHF_COORD_F64) {
    f[0] = wrap_fix(fixcoord_from_double(__ldg((const double*)p.x + i), frac) - cfix[0], boxfix);
    f[1] = wrap_fix(fixcoord_from_double(__ldg((const double*)p.y + i), frac) - cfix[1], boxfix);
    f[2] = wrap_fix(fixcoord_from_double(__ldg((const double*)p.z + i), frac) - cfix[2], boxfix);
  } else {
    f[0] = wrap_fix(fixcoord_from_float(__ldg((const float*)p.x + i), frac) - cfix[0], boxfix);
    f[1] = wrap_fix(fixcoord_from_float(__ldg((const float*)p.y + i), frac) - cfix[1], boxfix);
    f[2] = wrap_fix(fixcoord_from_float(__ldg((const float*)p.z + i), frac) - cfix[2], boxfix);
  }
}

// f * 2^-frac rounded to float (exact scaling of the correctly rounded integer).
__device__ __forceinline__ float f32_from_fixcoord(long long f, int frac) {
  return scale_pow2f(f32_from_i64_rn(f), -frac);
}

template <int CT>
__device__ __forceinline__ void load_velocity(const ParticlesDev& p, long long i, float v[3]) {
  if (CT == AHF_COORD_F64) {
    v[0] = (float)__ldg((const double*)p.vx + i);
    v[1] = (float)__ldg((const double*)p.vy + i);
    v[2] = (float)__ldg((const double*)p.vz + i);
  } else {
    v[0] = __ldg((const float*)p.vx + i);
    v[1] = __ldg((const float*)p.vy + i);
    v[2] = __ldg((const float*)p.vz + i);
  }
}

template <int CT>
__device__ __forceinline__ float load_mass(const ParticlesDev& p, long long i) {
  if (p.m == nullptr) return p.m0f;
  if (CT == AHF_COORD_F64) return (float)__ldg((const double*)p.m + i);
  return __ldg((const float*)p.m + i);
}

// Offset d = x - c of candidate i from the halo centre, rounded once to
// float.  With float inputs, no periodic box and a float-exact centre the
// IEEE subtraction already is that correctly rounded offset; otherwise the
// exact fixed-point route above.  Returns the fixed-point offset in f (valid
// only on the second route).
template <int CT>
__device__ __forceinline__ void offset_of(const ParticlesDev& p, long long i, const HaloDev& H, float d[3],
                                          long long f[3]) {
  if (CT != AHF_COORD_F64 && H.fast) {
    d[0] = __fsub_rn(__ldg((const float*)p.x + i), H.cf[0]);
    d[1] = __fsub_rn(__ldg((const float*)p.y + i), H.cf[1]);
    d[2] = __fsub_rn(__ldg((const float*)p.z + i), H.cf[2]);
  } else {
    load_offset_fix<CT>(p, i, H.cfix, H.boxfix, H.frac, f);
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = f32_from_fixcoord(f[k], H.frac);
  }
}

// Ask the copy engine to bring bytes [begin, end) of an array into L2
// (cp.async.bulk.prefetch, 16-byte granules): the range is rounded inwards,
// so nothing outside the array is named.  A hint only; it returns at once.
__device__ __forceinline__ void prefetch_l2(const void* base, unsigned long long begin, unsigned long long end) {
  unsigned long long a = ((unsigned long long)base + begin + 15ull) & ~15ull;
  const unsigned long long e = ((unsigned long long)base + end) & ~15ull;
  while (a < e) {
    const unsigned long long n = e - a < (1ull << 20) ? e - a : (1ull << 20);
    unsigned long long g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(a));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"((unsigned)n) : "memory");
    a += n;
  }
}

// Thread t < 8 of a group prefetches one input array over candidate slots
// [lo, hi) of a halo: the member list when there is one (the particles are
// then scattered), else the coordinate, velocity and mass arrays.
template <int CT>
__device__ __forceinline__ void prefetch_candidates(const ParticlesDev& p, const long long* member_idx, long long lo,
                                                    long long hi, int t) {
  if (t >= 8 || hi <= lo) return;
  if (member_idx) {
    if (t == 0) prefetch_l2(member_idx, 8ull * lo, 8ull * hi);
    return;
  }
  const void* arr[8] = {p.x, p.y, p.z, p.vx, p.vy, p.vz, p.m, nullptr};
  const unsigned long long es = CT == AHF_COORD_F64 ? 8ull : 4ull;
  if (arr[t]) prefetch_l2(arr[t], es * lo, es * hi);
}

// ---- radial sort of one CTA's (or one warp's) candidates ----------------------

// Shared-memory position of element p when each thread holds mask + 1
// consecutive elements: conflict-free for per-thread runs and warp stripes.
__device__ __forceinline__ int run_swizzle(int p, int mask) { return p ^ ((p >> 5) & mask); }

// 32-bit words of shared memory count_sort needs for NT threads (counters,
// then segment bases).
__host__ __device__ constexpr int count_sort_words(int nt) { return 8 * nt + 2 * nt; }

template <int NT>
__device__ __forceinline__ void group_sync() {
  if constexpr (NT == 32) __syncwarp();
  else __syncthreads();
}

// Stable LSD radix sort, 5-bit digits, of n (key, value) pairs held by NT
// threads (a CTA, or one warp for NT = 32) in runs: thread t holds positions
// [t ipt, t ipt + ipt) at run_swizzle(p, mask), ipt = mask + 1 <= IPT.  Only
// the bits of `diff` (keys agree elsewhere) are sorted.  Keys equal to
// KEY_NONMEMBER become `sub` on the way (a key above every member's, so that
// the non-members do not widen the digit range).
//
// Ranking is by counting, not by matching lanes: every thread counts the
// digits of its run in its own byte counters (word row*NT + t, row = digit &
// 7, byte = digit >> 3: conflict-free), one exclusive scan over the counters
// in (row, thread) order, four bytes at once, gives every (digit, thread)
// its first position.  The order is digit-major because a byte holds the
// digit's high part.  Ties keep their run order: the sort is stable.
// Returns 0 if the result is in (kA, vA), 1 if in (kB, vB).
template <int NT, int IPT>
__device__ int count_sort(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, uint32_t* aux, uint32_t* wtot,
                          int n, int mask, uint32_t diff, uint32_t sub, int t) {
  static_assert(IPT <= 16 && IPT % 4 == 0, "byte counters hold at most 16 per thread");
  if (diff == 0u) return 0;
  const int lo = __ffs(diff) - 1, hi = 31 - __clz(diff);
  const int ipt = mask + 1;
  const int lane = t & 31;
  uint32_t* cnt = aux;                                   // [8][NT] byte counters
  uint2* seg = reinterpret_cast<uint2*>(aux + 8 * NT);   // [NT] bases of 8-word segments
  uint32_t *kin = kA, *vin = vA, *kout = kB, *vout = vB;
  const int base = t * ipt;
  for (int shift = lo; shift <= hi; shift += 5) {
    // count (each thread touches only its own counters here)
#pragma unroll
    for (int w = 0; w < 8; ++w) cnt[w * NT + t] = 0u;
    uint32_t rk[IPT / 4];                                // rank among the run's equal digits
#pragma unroll
    for (int i = 0; i < IPT / 4; ++i) rk[i] = 0u;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      if (k < ipt && base + k < n) {
        const int q = run_swizzle(base + k, mask);
        uint32_t key = kin[q];
        if (shift == lo && key == KEY_NONMEMBER) {
          key = sub;
          kin[q] = key;
        }
        const uint32_t v = (key >> shift) & 31u;
        const int wi = (int)(v & 7u) * NT + t;
        const uint32_t sh = 8u * (v >> 3);
        const uint32_t c = cnt[wi];
        rk[k >> 2] |= ((c >> sh) & 0xffu) << (8 * (k & 3));
        cnt[wi] = c + (1u << sh);
      }
    }
    group_sync<NT>();
    // rake: thread t scans counter words [8t, 8t + 8) (in (row, thread)
    // order), leaving exclusive prefixes; bytes stay below 8 * 16
    uint4* c4 = reinterpret_cast<uint4*>(cnt) + 2 * t;
    const uint4 x0 = c4[0], x1 = c4[1];
    uint32_t s = 0;
    uint4 y0, y1;
    y0.x = s; s += x0.x; y0.y = s; s += x0.y; y0.z = s; s += x0.z; y0.w = s; s += x0.w;
    y1.x = s; s += x1.x; y1.y = s; s += x1.y; y1.z = s; s += x1.z; y1.w = s; s += x1.w;
    c4[0] = y0;
    c4[1] = y1;
    // exclusive scan of the segment sums over the threads, in 16-bit lanes:
    // a holds bytes 0 and 2, b bytes 1 and 3
    const uint32_t a = (s & 0xffu) | (((s >> 16) & 0xffu) << 16);
    const uint32_t b = ((s >> 8) & 0xffu) | (((s >> 24) & 0xffu) << 16);
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t xa = __shfl_up_sync(FULL_MASK, ia, o), xb = __shfl_up_sync(FULL_MASK, ib, o);
      if (lane >= o) {
        ia += xa;
        ib += xb;
      }
    }
    uint32_t ta, tb, pa = 0u, pb = 0u;
    if constexpr (NT == 32) {
      ta = __shfl_sync(FULL_MASK, ia, 31);
      tb = __shfl_sync(FULL_MASK, ib, 31);
    } else {
      const int warp = t >> 5;
      if (lane == 31) {
        wtot[2 * warp] = ia;
        wtot[2 * warp + 1] = ib;
      }
      __syncthreads();
      ta = 0u;
      tb = 0u;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) {
        const uint32_t xa = wtot[2 * w], xb = wtot[2 * w + 1];
        if (w < warp) {
          pa += xa;
          pb += xb;
        }
        ta += xa;
        tb += xb;
      }
    }
    // digit-major: the high part (byte) 0 first, then 1, 2, 3
    const uint32_t t0 = ta & 0xffffu, t1 = tb & 0xffffu, t2 = ta >> 16;
    seg[t] = make_uint2(pa + ia - a + ((t0 + t1) << 16), pb + ib - b + (t0 | ((t0 + t1 + t2) << 16)));
    group_sync<NT>();
    // scatter to the first position of (digit, thread) plus the run rank
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      if (k < ipt && base + k < n) {
        const int q = run_swizzle(base + k, mask);
        const uint32_t key = kin[q], val = vin[q];
        const uint32_t v = (key >> shift) & 31u;
        const int wi = (int)(v & 7u) * NT + t;
        const uint32_t hi2 = v >> 3;
        const uint2 sg = seg[wi >> 3];
        const uint32_t half = (hi2 & 1u) ? sg.y : sg.x;
        const uint32_t pos = ((half >> (16u * (hi2 >> 1))) & 0xffffu) + ((cnt[wi] >> (8u * hi2)) & 0xffu) +
                             ((rk[k >> 2] >> (8 * (k & 3))) & 0xffu);
        if (pos < (uint32_t)n) {               // always (a permutation of [0, n)); guards the store
          const int d = run_swizzle((int)pos, mask);
          kout[d] = key;
          vout[d] = val;
        }
      }
    }
    group_sync<NT>();
    uint32_t* tmp;
    tmp = kin; kin = kout; kout = tmp;
    tmp = vin; vin = vout; vout = tmp;
  }
  return kin == kA ? 0 : 1;
}

// Candidate records (OnchipLaunch::rec): written once by the gather, read
// back in radial order by the fill and the removals.  Plain (coherent)
// accesses: in a cluster another CTA may have written the record, which the
// cluster barrier between gather and fill (release / acquire) makes visible.
__device__ __forceinline__ void put_record(float4* r, const float d[3], float m, const float v[3]) {
  r[0] = make_float4(d[0], d[1], d[2], m);
  r[1] = make_float4(v[0], v[1], v[2], 0.0f);
}
__device__ __forceinline__ void get_record(const float4* r, float d[3], float& m, float v[3]) {
  const float4 a = r[0], b = r[1];
  d[0] = a.x; d[1] = a.y; d[2] = a.z; m = a.w;
  v[0] = b.x; v[1] = b.y; v[2] = b.z;
}
__device__ __forceinline__ void get_velocity_record(const float4* r, float v[3]) {
  const float4 b = r[1];
  v[0] = b.x; v[1] = b.y; v[2] = b.z;
}

// One candidate's stored fields, loaded together so that a loop can issue
// the loads of several candidates before using any of them (the particle
// store is read-only for the whole call).
template <int CT>
struct Cand {
  using E = typename std::conditional<CT == AHF_COORD_F64, double, float>::type;
  E x, y, z, vx, vy, vz, m;
};

template <int CT>
__device__ __forceinline__ void load_cand(const ParticlesDev& p, long long i, Cand<CT>& c) {
  using E = typename Cand<CT>::E;
  c.x = __ldg((const E*)p.x + i);
  c.y = __ldg((const E*)p.y + i);
  c.z = __ldg((const E*)p.z + i);
  c.vx = __ldg((const E*)p.vx + i);
  c.vy = __ldg((const E*)p.vy + i);
  c.vz = __ldg((const E*)p.vz + i);
  c.m = p.m ? __ldg((const E*)p.m + i) : (E)0;
}

template <int CT>
__device__ __forceinline__ float cand_mass(const ParticlesDev& p, const Cand<CT>& c) {
  return p.m ? (float)c.m : p.m0f;
}

template <int CT>
__device__ __forceinline__ void cand_velocity(const Cand<CT>& c, float v[3]) {
  v[0] = (float)c.vx;
  v[1] = (float)c.vy;
  v[2] = (float)c.vz;
}

// offset_of from loaded fields (same arithmetic, same result).
template <int CT>
__device__ __forceinline__ void cand_offset(const Cand<CT>& c, const HaloDev& H, float d[3], long long f[3]) {
  if (CT != AHF_COORD_F64 && H.fast) {
    d[0] = __fsub_rn((float)c.x, H.cf[0]);
    d[1] = __fsub_rn((float)c.y, H.cf[1]);
    d[2] = __fsub_rn((float)c.z, H.cf[2]);
  } else {
    if (CT == AHF_COORD_F64) {
      f[0] = wrap_fix(fixcoord_from_double((double)c.x, H.frac) - H.cfix[0], H.boxfix);
      f[1] = wrap_fix(fixcoord_from_double((double)c.y, H.frac) - H.cfix[1], H.boxfix);
      f[2] = wrap_fix(fixcoord_from_double((double)c.z, H.frac) - H.cfix[2], H.boxfix);
    } else {
      f[0] = wrap_fix(fixcoord_from_float((float)c.x, H.frac) - H.cfix[0], H.boxfix);
      f[1] = wrap_fix(fixcoord_from_float((float)c.y, H.frac) - H.cfix[1], H.boxfix);
      f[2] = wrap_fix(fixcoord_from_float((float)c.z, H.frac) - H.cfix[2], H.boxfix);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = f32_from_fixcoord(f[k], H.frac);
  }
}

// member_of from loaded fields (same decision).
template <int CT>
__device__ __forceinline__ bool cand_member(const Cand<CT>& c, const HaloDev& H, const float df[3],
                                            const long long f[3]) {
  const float r2f = fmaf(df[2], df[2], fmaf(df[1], df[1], df[0] * df[0]));
  if (r2f < H.R2lo) return true;
  if (r2f > H.R2hi) return false;
  double dd[3];
  if (CT != AHF_COORD_F64 && H.fast) {
    dd[0] = (double)(float)c.x - (double)H.cf[0];
    dd[1] = (double)(float)c.y - (double)H.cf[1];
    dd[2] = (double)(float)c.z - (double)H.cf[2];
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) dd[k] = scale_pow2d((double)f[k], -H.frac);
  }
  return dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2] <= H.R2;
}

// Member of the gather sphere: |d| <= R decided in FP64 arithmetic.  The
// float test settles all but the candidates within ~1e-6 of the surface.
__device__ __forceinline__ bool inside_sphere(const long long f[3], const float df[3], int frac, double R2,
                                              float R2lo, float R2hi) {
  const float r2f = fmaf(df[2], df[2], fmaf(df[1], df[1], df[0] * df[0]));
  if (r2f < R2lo) return true;
  if (r2f > R2hi) return false;
  double dd[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dd[k] = scale_pow2d((double)f[k], -frac);
  const double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
  return r2 <= R2;
}

// Membership of the candidate whose offset offset_of returned (FP64 decision).
template <int CT>
__device__ __forceinline__ bool member_of(const ParticlesDev& p, long long i, const HaloDev& H, const float df[3],
                                          const long long f[3]) {
  const float r2f = fmaf(df[2], df[2], fmaf(df[1], df[1], df[0] * df[0]));
  if (r2f < H.R2lo) return true;
  if (r2f > H.R2hi) return false;
  double dd[3];
  if (CT != AHF_COORD_F64 && H.fast) {
    // exact in FP64: the difference of two floats of similar magnitude
    dd[0] = (double)__ldg((const float*)p.x + i) - (double)H.cf[0];
    dd[1] = (double)__ldg((const float*)p.y + i) - (double)H.cf[1];
    dd[2] = (double)__ldg((const float*)p.z + i) - (double)H.cf[2];
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) dd[k] = scale_pow2d((double)f[k], -H.frac);
  }
  return dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2] <= H.R2;
}

__device__ __forceinline__ float radius_of(const float df[3]) {
  return sqrtf(fmaf(df[2], df[2], fmaf(df[1], df[1], df[0] * df[0])));
}

// m / max(r, r_soft) as the method's per-particle outer-sum term, and the
// reciprocal radius it uses.  r' = 0 contributes nothing (pairs at zero
// separation are dropped).
__device__ __forceinline__ float rinv_of(float r, float r_soft) {
  const float rr = fmaxf(r, r_soft);
  return rr > 0.0f ? __frcp_rn(rr) : 0.0f;
}

// phi_i = -G [M(<r_i) / r_i + sum_{j>=i} m_j / r_j] (Appendix A) from the
// float values of the inner mass, 1/r and the outer sum, rounded the same
// way in every kernel (explicit FMA: no compiler contraction choices).
__device__ __forceinline__ float phi_of(float m_inner, float rinv, float outer, float G) {
  return __fmul_rn(-G, __fmaf_rn(m_inner, rinv, outer));
}

// r <= e for a float radius r against the FP64 edge e (ef its float
// rounding), decided exactly.
__device__ __forceinline__ bool le_edge(float r, float ef, double e) {
  if (r < ef) return true;
  if (r > ef) return false;
  return (double)r <= e;
}

// Profile columns from the per-bin tables (see profile_bin_tables; tf is
// their float copy): the shell density M_bin / V_bin with V_bin = r_out^3
// (4 pi / 3)(f_{b+1}^3 - f_b^3), and v_circ = sqrt(G M(<= e_{b+1}) / e_{b+1}) with
// e_{b+1} = r_out f_{b+1}.  Both are formed in float (relative precision
// ~1e-7; counts and masses stay exact), in FP64 only if float overflows.
__device__ __forceinline__ double shell_density(double m_bin, double r_out, float inv_r, const double* tab,
                                                const float* tf, int n, int b) {
  const float d = ((double_to_float(m_bin) * (inv_r * inv_r * inv_r)) * tf[n + b]);
  if (isfinite(d) && (d > 0.0f || m_bin == 0.0)) return float_to_double(d);
  const double ir = 1.0 / r_out;
  return (m_bin * (ir * ir * ir)) * tab[n + b];
}
__device__ __forceinline__ double circular_velocity(double G, float Gf, double m_in, double r_out, float inv_r,
                                                    const double* tab, const float* tf, int n, int b) {
  const float v2 = ((Gf * double_to_float(m_in)) * inv_r) * tf[2 * n + b];
  if (isfinite(v2) && (v2 > 0.0f || m_in == 0.0)) return float_to_double(sqrtf(v2));
  return sqrt(((G * m_in) / r_out) * tab[2 * n + b]);
}

// r <= e for a float radius r and the FP64 edge e = r_out fac, decided against
// ef = r_out_f fac_f (float values within three roundings of e) outside an
// 8-ulp band, in FP64 inside it.
__device__ __forceinline__ bool le_edge_band(float r, float ef, double r_out, double fac) {
  if (r < ef * (1.0f - 4.8e-7f)) return true;
  if (r > ef * (1.0f + 4.8e-7f)) return false;
  return float_to_double(r) <= r_out * fac;
}

// Log-radial profile rows of one halo from its compacted bound set held on
// chip: radii rc[idx(k)] ascending and inclusive exact masses mc[idx(k)]
// (scale 2^-s_m), k < nb.  Row b covers (e_b, e_{b+1}], e_b = r_out f^(1-b/n),
// r_out = r_vir or the outermost bound radius (Sect. 2.1, the radially binned
// output).  The calling threads take rows t0, t0 + stride, ...
template <typename Idx>
__device__ void profile_rows(const ProfileRows& Q, int h, const float* rc, const long long* mc, Idx idx, long long nb,
                             double r_vir, int s_m, double G, float Gf, const double* m0, int t0, int stride) {
  const int n = Q.n_bins;
  double* out = Q.prof + (size_t)h * n * 4;
  if (nb == 0) {
    for (int i = t0; i < 4 * n; i += stride) out[i] = 0.0;
    return;
  }
  const double r_out = r_vir > 0.0 ? r_vir : float_to_double(rc[idx(nb - 1)]);
  const float r_out_f = double_to_float(r_out);
  const float inv_r = 1.0f / r_out_f;
  auto count_le = [&](int b) {               // first k with rc[k] > e_b (b = n: r_out)
    const float ef = b == n ? r_out_f : r_out_f * Q.factor_f[b];
    const double fac = b == n ? 1.0 : Q.factor[b];
    long long lo = 0, hi = nb;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (le_edge_band(rc[idx(mid)], ef, r_out, fac)) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  for (int b = t0; b < n; b += stride) {
    const long long c0 = count_le(b), c1 = count_le(b + 1);
    // masses: count * m0 for a uniform particle mass (m0 != NULL), else the
    // exact fixed-point sums
    double M1, Mshell;
    if (m0) {
      M1 = double_from_fix(c1, 0) * *m0;
      Mshell = double_from_fix(c1 - c0, 0) * *m0;
    } else {
      const long long f0 = c0 > 0 ? mc[idx(c0 - 1)] : 0;
      const long long f1 = c1 > 0 ? mc[idx(c1 - 1)] : 0;
      M1 = double_from_fix(f1, s_m);
      Mshell = double_from_fix(f1 - f0, s_m);
    }
    out[4 * b + 0] = double_from_fix(c1 - c0, 0);
    out[4 * b + 1] = M1;
    out[4 * b + 2] = shell_density(Mshell, r_out, inv_r, Q.factor, Q.factor_f, n, b);
    out[4 * b + 3] = circular_velocity(G, Gf, M1, r_out, inv_r, Q.factor, Q.factor_f, n, b);
  }
}

// ---- per-halo trace (AHF_OPT_TRACE) ------------------------------------------------

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int sm_id() {
  int s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

// Record trace field f of halo h (no-op when tracing is off).
__device__ __forceinline__ void trace_mark(long long* trace, int h, int f) {
  if (trace) trace[(size_t)h * AHF_TRACE_FIELDS + f] = global_ns();
}

// ---- warp / block scans ---------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
  return x;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace ahf
