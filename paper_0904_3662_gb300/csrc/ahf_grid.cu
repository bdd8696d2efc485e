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

// ---- prepare ---------------------------------------------------------------------

template <int CT>
__global__ void __launch_bounds__(T) g_prepare(GridLaunch L) {
  const int t = blockIdx.x;
  const int2 tr = L.tile_range[t];
  const int k = L.tile_halo[t];
  const HaloDev H = L.halos[k];
  const ParamsDev& P = L.prm;
  uint32_t orb = 0u, andb = 0xffffffffu, mxm = 0u, mxr = 0u, mxv = 0u;
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
    uint32_t key = KEY_NONMEMBER;
    if (ok) {
      long long f[3];
      load_offset_fix<CT>(L.p, pi, H.cfix, H.boxfix, H.frac, f);
      float df[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) df[a] = f32_from_fixcoord(f[a], H.frac);
      if (inside_sphere(f, df, H.frac, H.R2, H.R2lo, H.R2hi)) {
        const float r = radius_of(df);
        key = __float_as_uint(r);
        const float m = load_mass<CT>(L.p, pi);
        float v[3];
        load_velocity<CT>(L.p, pi, v);
        mxm = max(mxm, __float_as_uint(fabsf(m)));
        mxr = max(mxr, __float_as_uint(fabsf(m * rinv_of(r, P.r_soft_f))));
#pragma unroll
        for (int a = 0; a < 3; ++a) mxv = max(mxv, __float_as_uint(fabsf(__fmul_rn(m, v[a]))));
        ++nmem;
      }
    }
    if (key == KEY_NONMEMBER && L.out.removed_iter) L.out.removed_iter[slot] = -1;
    L.key_a[g] = key;
    L.val_a[g] = (uint32_t)i;
    orb |= key;
    andb &= key;
  }
  orb = __reduce_or_sync(FULL_MASK, orb);
  andb = __reduce_and_sync(FULL_MASK, andb);
  mxm = __reduce_max_sync(FULL_MASK, mxm);
  mxr = __reduce_max_sync(FULL_MASK, mxr);
  mxv = __reduce_max_sync(FULL_MASK, mxv);
  nmem = __reduce_add_sync(FULL_MASK, nmem);
  if ((threadIdx.x & 31) == 0) {
    GridHaloState* s = L.state + k;
    atomicOr(&L.key_or_and[0], orb);
    atomicAnd(&L.key_or_and[1], andb);
    atomicMax(&s->mass_max_bits, (unsigned long long)mxm);
    atomicMax(&s->mr_max_bits, (unsigned long long)mxr);
    atomicMax(&s->mv_max_bits, (unsigned long long)mxv);
    if (nmem) atomicAdd((unsigned long long*)&s->n_member, (unsigned long long)nmem);
  }
}

__global__ void g_scales(GridLaunch L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.n_halos) return;
  GridHaloState& s = L.state[k];
  const long long n = s.n_member;
  s.s_m = fix_scale(float_exponent_of_bits((uint32_t)s.mass_max_bits), n);
  s.s_mr = fix_scale(float_exponent_of_bits((uint32_t)s.mr_max_bits), n);
  s.s_mv = fix_scale(float_exponent_of_bits((uint32_t)s.mv_max_bits), n);
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
__global__ void __launch_bounds__(T) g_hist(const uint32_t* __restrict__ key, const int2* __restrict__ tile_range,
                                            const int* __restrict__ tile_halo, const int* __restrict__ halo_tile0,
                                            uint32_t* __restrict__ tile_hist, int shift) {
  __shared__ uint32_t h[256];
  const int t = blockIdx.x;
  const int2 tr = tile_range[t];
  const int k = tile_halo[t];
  const int t0 = halo_tile0[k], th = halo_tile0[k + 1] - t0;
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < tr.y; e += T) atomicAdd(&h[(key[tr.x + e] >> shift) & 0xffu], 1u);
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

__global__ void __launch_bounds__(T) g_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
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
  uint32_t key[IPT], val[IPT];
  uint16_t rank[IPT];
#pragma unroll
  for (int b = 0; b < IPT; ++b) {
    const int e = warp * CH + b * 32 + lane;
    const bool valid = e < tr.y;
    key[b] = valid ? kin[tr.x + e] : 0u;
    val[b] = valid ? vin[tr.x + e] : 0u;
    const unsigned vmask = __ballot_sync(FULL_MASK, valid);
    rank[b] = 0;
    if (valid) {
      const uint32_t dg = (key[b] >> shift) & 0xffu;
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
      const uint32_t dg = (key[b] >> shift) & 0xffu;
      const long long dst = gb + (long long)doff[dg] + hist[warp * 256 + dg] + rank[b];
      kout[dst] = key[b];
      vout[dst] = val[b];
    }
  }
}

// ---- fill -------------------------------------------------------------------------

template <int CT>
__global__ void __launch_bounds__(T) g_fill(GridLaunch L, const uint32_t* __restrict__ key,
                                            const uint32_t* __restrict__ val) {
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
      long long f[3];
      load_offset_fix<CT>(L.p, pi, H.cfix, H.boxfix, H.frac, f);
      float v[3];
      load_velocity<CT>(L.p, pi, v);
      const float m = load_mass<CT>(L.p, pi);
      float4 w;
      w.x = fmaf(L.prm.Hf, f32_from_fixcoord(f[0], H.frac), v[0]);
      w.y = fmaf(L.prm.Hf, f32_from_fixcoord(f[1], H.frac), v[1]);
      w.z = fmaf(L.prm.Hf, f32_from_fixcoord(f[2], H.frac), v[2]);
      w.w = m;
      L.wm[g] = w;
      L.r[g] = __uint_as_float(key[g]);
#pragma unroll
      for (int a = 0; a < 3; ++a) smv[a] += fix_from_float(__fmul_rn(m, v[a]), s_v);
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
__global__ void __launch_bounds__(T) g_tile_sums(GridLaunch L, int final_pass) {
  const int t = blockIdx.x;
  const int k = L.tile_halo[t];
  const GridHaloState& S = L.state[k];
  if (!final_pass && !S.active) return;
  const int2 tr = L.tile_range[t];
  const long long lim = L.halos[k].gbase + S.n_member;
  long long a = 0, b = 0, c = 0;
  const int s_m = S.s_m, s_r = S.s_mr;
  const float rs = L.prm.r_soft_f;
  for (int e = threadIdx.x; e < tr.y; e += T) {
    const long long g = (long long)tr.x + e;
    if (g < lim) {
      const float m = L.wm[g].w;
      if (!signbit(m)) {
        a += fix_from_float(m, s_m);
        b += fix_from_float(m * rinv_of(L.r[g], rs), s_r);
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
      const float mt = float_from_fix(carry[0], S.s_m);
      for (int a = 0; a < 3; ++a) S.vbulk[a] = float_from_fix(S.mv[a], S.s_mv) / mt;
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

template <int CT>
__global__ void __launch_bounds__(T) g_apply(GridLaunch L, int iter) {
  const int t = blockIdx.x;
  const int k = L.tile_halo[t];
  GridHaloState& S = L.state[k];
  if (!S.active) return;
  const int2 tr = L.tile_range[t];
  const HaloDev& H = L.halos[k];
  const long long lim = H.gbase + S.n_member;
  const int s_m = S.s_m, s_r = S.s_mr, s_v = S.s_mv;
  const ParamsDev& P = L.prm;
  const float vb0 = S.vbulk[0], vb1 = S.vbulk[1], vb2 = S.vbulk[2];
  const long long Ttot = S.t_tot;
  const long long g0 = (long long)tr.x + (long long)threadIdx.x * IPT;
  // pass 1: thread totals over its IPT consecutive elements
  float4 wmv[IPT];
  float rv[IPT];
  long long a = 0, b = 0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const long long g = g0 + q;
    const bool in = (threadIdx.x * IPT + q < tr.y) && g < lim;
    wmv[q] = in ? L.wm[g] : make_float4(0.f, 0.f, 0.f, -0.0f);
    rv[q] = in ? L.r[g] : 1.0f;
    if (!signbit(wmv[q].w)) {
      a += fix_from_float(wmv[q].w, s_m);
      b += fix_from_float(wmv[q].w * rinv_of(rv[q], P.r_soft_f), s_r);
    }
  }
  TileScan ts = block_scan_tile(a, b, 0, L.tile_pre[(size_t)t * 3 + 0], L.tile_pre[(size_t)t * 3 + 1], 0);
  long long M = ts.m, Pp = ts.r;
  long long rm = 0, rv0 = 0, rv1 = 0, rv2 = 0;
  int nrem = 0, nband = 0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const float m = wmv[q].w;
    if (!signbit(m)) {
      const float ri = rinv_of(rv[q], P.r_soft_f);
      const long long mfix = fix_from_float(m, s_m);
      const long long rfix = fix_from_float(m * ri, s_r);
      const float phi = phi_of(float_from_fix(M, s_m), ri, float_from_fix(Ttot - Pp, s_r), P.Gf);
      const float ux = wmv[q].x - vb0, uy = wmv[q].y - vb1, uz = wmv[q].z - vb2;
      const float u2 = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
      const float two_phi = -2.0f * phi;
      if (fabsf(u2 - two_phi) < P.band_f * two_phi) ++nband;
      if (u2 > two_phi) {
        const long long g = g0 + q;
        L.wm[g].w = -m;
        ++nrem;
        const long long slot = H.offset + L.val_x[g];
        const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
        float v[3];
        load_velocity<CT>(L.p, pi, v);
        rm += mfix;
        rv0 += fix_from_float(__fmul_rn(m, v[0]), s_v);
        rv1 += fix_from_float(__fmul_rn(m, v[1]), s_v);
        rv2 += fix_from_float(__fmul_rn(m, v[2]), s_v);
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

__global__ void __launch_bounds__(T) g_emit(GridLaunch L) {
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
  float mq[IPT], rq[IPT];
  long long a = 0, b = 0, c = 0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const long long g = g0 + q;
    const bool in = (threadIdx.x * IPT + q < tr.y) && g < lim;
    mq[q] = in ? L.wm[g].w : -0.0f;
    rq[q] = in ? L.r[g] : 1.0f;
    if (!signbit(mq[q])) {
      a += fix_from_float(mq[q], s_m);
      b += fix_from_float(mq[q] * rinv_of(rq[q], P.r_soft_f), s_r);
      c += 1;
    }
  }
  const size_t tp = (size_t)t * 3;
  TileScan ts = block_scan_tile(a, b, c, L.tile_pre[tp], L.tile_pre[tp + 1], L.tile_pre[tp + 2]);
  long long M = ts.m, Pp = ts.r, C = ts.c;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const float m = mq[q];
    if (!signbit(m)) {
      const long long g = g0 + q;
      const float ri = rinv_of(rq[q], P.r_soft_f);
      const long long mfix = fix_from_float(m, s_m);
      const float phi = phi_of(float_from_fix(M, s_m), ri, float_from_fix(Ttot - Pp, s_r), P.Gf);
      const long long slot = H.offset + L.val_x[g];
      const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
      const long long dst = H.offset + C;
      L.out.bound_idx[dst] = pi;
      if (L.out.phi) ((float*)L.out.phi)[dst] = phi;
      if (L.out.removed_iter) L.out.removed_iter[slot] = 0;
      L.rc[H.gbase + C] = rq[q];
      L.mc[H.gbase + C] = M + mfix;
      M += mfix;
      Pp += fix_from_float(m * ri, s_r);
      C += 1;
    }
  }
}

// First compacted index k with M_k < delta_rho 4pi/3 r_{k+1}^3 (r_{N+1} = inf).
__global__ void __launch_bounds__(T) g_virial(GridLaunch L) {
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
      const float rn = L.rc[g + 1];
      const long long mk = L.mc[g];
      const float lhs = float_from_fix(mk, S.s_m);
      const float rhs = P.crit_f * rn * rn * rn;
      if (lhs < rhs * (1.0f - 1e-5f)) cross = true;
      else if (lhs > rhs * (1.0f + 1e-5f)) cross = false;
      else {
        const double rd = (double)rn;
        cross = double_from_fix(mk, S.s_m) < P.crit * rd * rd * rd;
      }
    }
    if (cross) { kf = kk; break; }
  }
  // warp min then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) kf = min(kf, __shfl_xor_sync(FULL_MASK, kf, o));
  if ((threadIdx.x & 31) == 0 && kf != 0x7fffffffffffffffll)
    atomicMin((unsigned long long*)&S.k_first, (unsigned long long)kf);
}

__global__ void g_result(GridLaunch L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.n_halos) return;
  const GridHaloState& S = L.state[k];
  const HaloDev& H = L.halos[k];
  ahf_result R;
  const long long nb = S.n_alive;
  R.n_bound = nb;
  R.n_member = S.n_member;
  R.part_iter = S.part_iter;
  R.n_band = S.band;
  R.n_iter = S.n_iter;
  R.k_vir = -1;
  R.m_vir = 0.0;
  R.r_vir = 0.0;
  int status = S.status;
  if (S.n_member == 0) status |= AHF_HALO_EMPTY;
  if (nb > 0) {
    const long long kk = S.k_first;
    const double mk = double_from_fix(L.mc[H.gbase + kk], S.s_m);
    const double rk = (double)L.rc[H.gbase + kk];
    if (kk == nb - 1) status |= AHF_HALO_RVIR_BEYOND_EDGE;
    if (mk < L.prm.crit * rk * rk * rk) {
      status |= AHF_HALO_RVIR_NONE;
    } else {
      R.k_vir = kk;
      R.m_vir = mk;
      R.r_vir = cbrt(mk / L.prm.crit);
    }
    const double mt = double_from_fix(S.m_tot, S.s_m);
    for (int a = 0; a < 3; ++a) R.vbulk[a] = double_from_fix(S.mv[a], S.s_mv) / mt;
  } else {
    R.vbulk[0] = R.vbulk[1] = R.vbulk[2] = 0.0;
  }
  R.status = status;
  L.out.res[H.index] = R;
}

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

}  // namespace

cudaError_t grid_prepare(const GridLaunch& L, cudaStream_t s) {
  if (L.p.coord_type == AHF_COORD_F64) g_prepare<AHF_COORD_F64><<<L.n_tiles, T, 0, s>>>(L);
  else g_prepare<AHF_COORD_F32_REL><<<L.n_tiles, T, 0, s>>>(L);
  g_scales<<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t grid_sort(GridLaunch& L, cudaStream_t s, uint32_t or_bits, uint32_t and_bits) {
  const uint32_t diff = or_bits ^ and_bits;
  uint32_t *ki = L.key_a, *vi = L.val_a, *ko = L.key_b, *vo = L.val_b;
  L.sort_passes = 0;
  for (int d = 0; d < 4; ++d) {
    if (!((diff >> (8 * d)) & 0xffu)) continue;
    ++L.sort_passes;
    const int shift = 8 * d;
    g_hist<<<L.n_tiles, T, 0, s>>>(ki, L.tile_range, L.tile_halo, L.halo_tile0, L.tile_hist, shift);
    g_digit_scan<<<L.n_halos * 256, 256, 0, s>>>(L.tile_hist, L.halo_tile0, L.digit_base);
    g_digit_base<<<L.n_halos, 256, 0, s>>>(L.digit_base);
    g_scatter<<<L.n_tiles, T, 0, s>>>(ki, vi, ko, vo, L.tile_range, L.tile_halo, L.halo_tile0, L.halos,
                                      L.tile_hist, L.digit_base, shift);
    uint32_t* x;
    x = ki; ki = ko; ko = x;
    x = vi; vi = vo; vo = x;
  }
  L.key_x = ki;
  L.val_x = vi;
  return cudaGetLastError();
}

cudaError_t grid_fill(const GridLaunch& L, cudaStream_t s) {
  if (L.p.coord_type == AHF_COORD_F64) g_fill<AHF_COORD_F64><<<L.n_tiles, T, 0, s>>>(L, L.key_x, L.val_x);
  else g_fill<AHF_COORD_F32_REL><<<L.n_tiles, T, 0, s>>>(L, L.key_x, L.val_x);
  return cudaGetLastError();
}

cudaError_t grid_iterate(const GridLaunch& L, int iter, cudaStream_t s) {
  g_tile_sums<<<L.n_tiles, T, 0, s>>>(L, 0);
  g_tile_scan<<<L.n_halos, 256, 0, s>>>(L, 0);
  if (L.p.coord_type == AHF_COORD_F64) g_apply<AHF_COORD_F64><<<L.n_tiles, T, 0, s>>>(L, iter);
  else g_apply<AHF_COORD_F32_REL><<<L.n_tiles, T, 0, s>>>(L, iter);
  g_advance<<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t grid_finish(const GridLaunch& L, cudaStream_t s) {
  g_tile_sums<<<L.n_tiles, T, 0, s>>>(L, 1);
  g_tile_scan<<<L.n_halos, 256, 0, s>>>(L, 1);
  g_emit<<<L.n_tiles, T, 0, s>>>(L);
  g_virial<<<L.n_tiles, T, 0, s>>>(L);
  g_result<<<blocks_for(L.n_halos, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace ahf
