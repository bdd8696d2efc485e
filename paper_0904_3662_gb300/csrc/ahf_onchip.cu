// On-chip class: one CTA unbinds one halo entirely in shared memory.
//
// Per halo (Sect. 2.1 and Appendix A):
//   gather   candidates -> (radius key, candidate position), FP64-accurate
//            recentring and sphere test, exponent maxima for the exact sums
//   sort     stable LSD radix sort of the keys in shared memory (once: the
//            centre is fixed and particles only leave, so the survivors of
//            every later iteration stay in radial order)
//   fill     sorted SoA: radius, mass, w = v + H d; exact sum m v
//   iterate  block scan of the exact M(<r) and sum m/r prefixes ->
//            phi_i = -G [M(<r_i)/r_i + sum_{j>=i} m_j/r_j], escape test
//            |w - v_bulk|^2 > 2|phi|, removal of every unbound particle, until
//            an iteration removes nothing
//   emit     bound list (particle index, phi) in radial order, virial crossing
//            of the final set (Sect. 2.1, Eqs. 1-2), result record
//
// CTAs are persistent: each pulls the next halo from a counter over the
// class's haloes, which the host orders largest first.
#include <cstdint>

#include "ahf_device.cuh"

namespace ahf {
namespace {

// Swizzled shared-memory position of element p for a blocked arrangement of
// ipt = mask + 1 consecutive elements per thread: conflict-free both for
// per-thread runs and for warp-striped access.
__device__ __forceinline__ int sw(int p, int mask) { return p ^ ((p >> 5) & mask); }

template <int NT>
struct Smem {
  static constexpr int NW = NT / 32;
  long long red[NW][4];          // per-warp partials (block scans / reductions)
  long long scan_base[NW][3];
  unsigned int or_bits, and_bits;
  unsigned int max_m, max_mr, max_mv;
  int n_member;
  long long mv[3];               // exact sum m v of the current set
  long long rem[4];              // removed this iteration: m, m v (3)
  long long tot[3];              // scan totals: M, sum m/r, count
  int removed;
  int band;
  int k_first;
  int halo;
  float vb[3];
  uint32_t dtot[256];            // radix sort digit totals / offsets
};

template <int NT>
__device__ __forceinline__ void block_exclusive_scan3(long long& a, long long& b, long long& c, Smem<NT>& S,
                                                      long long& ta, long long& tb, long long& tc) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long ia = warp_inclusive_scan(a, lane);
  long long ib = warp_inclusive_scan(b, lane);
  long long ic = warp_inclusive_scan(c, lane);
  if (lane == 31) { S.red[warp][0] = ia; S.red[warp][1] = ib; S.red[warp][2] = ic; }
  __syncthreads();
  if (warp == 0) {
    long long x = lane < NW ? S.red[lane][0] : 0, y = lane < NW ? S.red[lane][1] : 0,
              z = lane < NW ? S.red[lane][2] : 0;
    long long sx = warp_inclusive_scan(x, lane), sy = warp_inclusive_scan(y, lane), sz = warp_inclusive_scan(z, lane);
    if (lane < NW) { S.scan_base[lane][0] = sx - x; S.scan_base[lane][1] = sy - y; S.scan_base[lane][2] = sz - z; }
    if (lane == NW - 1) { S.tot[0] = sx; S.tot[1] = sy; S.tot[2] = sz; }
  }
  __syncthreads();
  a = S.scan_base[warp][0] + ia - a;
  b = S.scan_base[warp][1] + ib - b;
  c = S.scan_base[warp][2] + ic - c;
  ta = S.tot[0]; tb = S.tot[1]; tc = S.tot[2];
}

// Stable LSD radix sort of n (key, val) pairs, 8-bit digits, skipping the
// digits in which all keys agree.  The last pass writes element p at
// sw(p, mask).  Returns 0 if the result is in (kA, vA), 1 if in (kB, vB).
template <int NT, int IPT>
__device__ int block_radix_sort(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, uint16_t* hist,
                                uint32_t* dtot, int n, uint32_t diff, int mask) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int passes[4], np = 0;
  for (int d = 0; d < 4; ++d)
    if ((diff >> (8 * d)) & 0xffu) passes[np++] = d;
  uint32_t *kin = kA, *vin = vA, *kout = kB, *vout = vB;
  if (np == 0) {
    for (int p = threadIdx.x; p < n; p += NT) {
      kB[sw(p, mask)] = kA[p];
      vB[sw(p, mask)] = vA[p];
    }
    __syncthreads();
    return 1;
  }
  const int chunk = ((n + NW * 32 - 1) / (NW * 32)) * 32;      // per-warp run
  const int nb = chunk / 32;                                   // <= IPT
  for (int ip = 0; ip < np; ++ip) {
    const int shift = 8 * passes[ip];
    const bool last = (ip == np - 1);
    for (int i = threadIdx.x; i < NW * 256; i += NT) hist[i] = 0;
    __syncthreads();
    uint32_t key[IPT], val[IPT];
    uint16_t rank[IPT];
#pragma unroll
    for (int b = 0; b < IPT; ++b) {
      if (b < nb) {
        const int e = warp * chunk + b * 32 + lane;
        const bool valid = e < n;
        key[b] = valid ? kin[e] : 0u;
        val[b] = valid ? vin[e] : 0u;
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
    }
    __syncthreads();
    // digit-major, warp-minor exclusive offsets: digit totals, one warp scans
    // them, then each digit's per-warp counts become running offsets
    for (int dg = threadIdx.x; dg < 256; dg += NT) {
      uint32_t tot = 0;
      for (int w = 0; w < NW; ++w) tot += hist[w * 256 + dg];
      dtot[dg] = tot;
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t loc[8], s = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { loc[i] = dtot[lane * 8 + i]; s += loc[i]; }
      const uint32_t inc = warp_inclusive_scan(s, lane);
      uint32_t run = inc - s;
#pragma unroll
      for (int i = 0; i < 8; ++i) { dtot[lane * 8 + i] = run; run += loc[i]; }
    }
    __syncthreads();
    for (int dg = threadIdx.x; dg < 256; dg += NT) {
      uint32_t run = dtot[dg];
      for (int w = 0; w < NW; ++w) {
        const uint32_t h = hist[w * 256 + dg];
        hist[w * 256 + dg] = (uint16_t)run;
        run += h;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < IPT; ++b) {
      if (b < nb) {
        const int e = warp * chunk + b * 32 + lane;
        if (e < n) {
          const uint32_t dg = (key[b] >> shift) & 0xffu;
          int dst = (int)hist[warp * 256 + dg] + (int)rank[b];
          if (last) dst = sw(dst, mask);
          kout[dst] = key[b];
          vout[dst] = val[b];
        }
      }
    }
    __syncthreads();
    uint32_t* t;
    t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
  }
  return (kin == kA) ? 0 : 1;
}

template <int NT>
constexpr int min_blocks() { return NT <= 128 ? 8 : (NT <= 256 ? 2 : 1); }

template <int NT, int CAP, int CT>
__global__ void __launch_bounds__(NT, min_blocks<NT>()) onchip_kernel(OnchipLaunch L) {
  constexpr int NW = NT / 32;
  constexpr int IPT = CAP / NT;
  static_assert(IPT * NT == CAP && IPT <= 32 && (IPT & (IPT - 1)) == 0, "bad tile");
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Smem<NT> S;
  uint32_t* kA = (uint32_t*)dyn;
  uint32_t* vA = kA + CAP;
  uint32_t* kB = vA + CAP;
  uint32_t* vB = kB + CAP;
  float* ex1 = (float*)(vB + CAP);
  float* ex2 = ex1 + CAP;
  uint16_t* hist = (uint16_t*)(ex2 + CAP);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const ParamsDev& P = L.prm;

  for (;;) {
    if (tid == 0) S.halo = atomicAdd(L.queue, 1);
    __syncthreads();
    const int hq = S.halo;
    if (hq >= L.n_halos) break;
    const HaloDev H = L.halos[hq];
    const int n_cand = (int)H.count;
    if (tid == 0) {
      S.or_bits = 0u; S.and_bits = 0xffffffffu;
      S.max_m = 0u; S.max_mr = 0u; S.max_mv = 0u;
      S.n_member = 0;
      S.mv[0] = S.mv[1] = S.mv[2] = 0;
    }
    __syncthreads();
    if (n_cand > CAP) {   // the scheduler never does this; report, do not overrun
      if (tid == 0) atomicOr(L.out.err, ERR_CAPACITY);
      __syncthreads();
      continue;
    }

    // ---- gather: key = radius bits of members, candidate position as value ----
    {
      uint32_t orb = 0u, andb = 0xffffffffu, mxm = 0u, mxr = 0u, mxv = 0u;
      int nmem = 0;
      for (int i = tid; i < n_cand; i += NT) {
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
          for (int k = 0; k < 3; ++k) df[k] = f32_from_fixcoord(f[k], H.frac);
          if (inside_sphere(f, df, H.frac, H.R2, H.R2lo, H.R2hi)) {
            const float r = radius_of(df);
            key = __float_as_uint(r);
            const float m = load_mass<CT>(L.p, pi);
            float v[3];
            load_velocity<CT>(L.p, pi, v);
            const float mr = m * rinv_of(r, P.r_soft_f);
            mxm = max(mxm, __float_as_uint(fabsf(m)));
            mxr = max(mxr, __float_as_uint(fabsf(mr)));
#pragma unroll
            for (int k = 0; k < 3; ++k) mxv = max(mxv, __float_as_uint(fabsf(__fmul_rn(m, v[k]))));
            ++nmem;
          }
        }
        if (key == KEY_NONMEMBER && L.out.removed_iter) L.out.removed_iter[slot] = -1;
        kA[i] = key;
        vA[i] = (uint32_t)i;
        orb |= key;
        andb &= key;
      }
      orb = __reduce_or_sync(FULL_MASK, orb);
      andb = __reduce_and_sync(FULL_MASK, andb);
      mxm = __reduce_max_sync(FULL_MASK, mxm);
      mxr = __reduce_max_sync(FULL_MASK, mxr);
      mxv = __reduce_max_sync(FULL_MASK, mxv);
      nmem = __reduce_add_sync(FULL_MASK, nmem);
      if (lane == 0) {
        atomicOr(&S.or_bits, orb);
        atomicAnd(&S.and_bits, andb);
        atomicMax(&S.max_m, mxm);
        atomicMax(&S.max_mr, mxr);
        atomicMax(&S.max_mv, mxv);
        atomicAdd(&S.n_member, nmem);
      }
    }
    __syncthreads();
    const int n_mem = S.n_member;
    int ipt = 1;
    while (ipt * NT < n_mem) ipt <<= 1;
    const int mask = ipt - 1;
    const int s_m = fix_scale(float_exponent_of_bits(S.max_m), n_mem);
    const int s_r = fix_scale(float_exponent_of_bits(S.max_mr), n_mem);
    const int s_v = fix_scale(float_exponent_of_bits(S.max_mv), n_mem);

    // ---- radial sort (once) ----
    const int which = block_radix_sort<NT, IPT>(kA, vA, kB, vB, hist, S.dtot, n_cand, S.or_bits ^ S.and_bits, mask);
    float* rr = (float*)(which ? kB : kA);         // radius, sorted, swizzled
    uint32_t* jj = which ? vB : vA;                // candidate position
    float* mm = (float*)(which ? kA : kB);         // mass; sign bit = removed
    float* wx = (float*)(which ? vA : vB);
    float* wy = ex1;
    float* wz = ex2;

    // ---- fill: sorted SoA and the exact sum m v of the members ----
    {
      long long smv[3] = {0, 0, 0};
      for (int p = tid; p < n_mem; p += NT) {
        const int q = sw(p, mask);
        const int j = (int)jj[q];
        const long long slot = H.offset + j;
        const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
        long long f[3];
        load_offset_fix<CT>(L.p, pi, H.cfix, H.boxfix, H.frac, f);
        float v[3];
        load_velocity<CT>(L.p, pi, v);
        const float m = load_mass<CT>(L.p, pi);
        mm[q] = m;
        wx[q] = fmaf(P.Hf, f32_from_fixcoord(f[0], H.frac), v[0]);
        wy[q] = fmaf(P.Hf, f32_from_fixcoord(f[1], H.frac), v[1]);
        wz[q] = fmaf(P.Hf, f32_from_fixcoord(f[2], H.frac), v[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) smv[k] += fix_from_float(__fmul_rn(m, v[k]), s_v);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const long long t = warp_sum(smv[k]);
        if (lane == 0) atomicAdd((unsigned long long*)&S.mv[k], (unsigned long long)t);
      }
    }
    __syncthreads();

    // ---- iterate (Appendix A) ----
    int n_iter = 0, status = 0;
    long long part_iter = 0, n_band = 0;
    int n_alive = n_mem;
    bool converged = false;
    const int p0 = tid * ipt;
    while (n_alive > 0 && n_iter < P.max_iter) {
      ++n_iter;
      part_iter += n_alive;
      // pass 1: per-thread exact sums of m and m/r over alive particles
      long long tm = 0, tr = 0, tc = 0;
      for (int k = 0; k < ipt; ++k) {
        const int p = p0 + k;
        if (p < n_mem) {
          const int q = sw(p, mask);
          const float m = mm[q];
          if (!signbit(m)) {
            tm += fix_from_float(m, s_m);
            tr += fix_from_float(m * rinv_of(rr[q], P.r_soft_f), s_r);
          }
        }
      }
      long long M_tot, T_tot, C_tot;
      block_exclusive_scan3<NT>(tm, tr, tc, S, M_tot, T_tot, C_tot);
      if (tid == 0) {
        // v_bulk = sum m v / sum m of the current set, from the exact sums
        const float mt = float_from_fix(M_tot, s_m);
        S.vb[0] = float_from_fix(S.mv[0], s_v) / mt;
        S.vb[1] = float_from_fix(S.mv[1], s_v) / mt;
        S.vb[2] = float_from_fix(S.mv[2], s_v) / mt;
        S.rem[0] = S.rem[1] = S.rem[2] = S.rem[3] = 0;
        S.removed = 0;
        S.band = 0;
      }
      __syncthreads();
      const float vb0 = S.vb[0], vb1 = S.vb[1], vb2 = S.vb[2];
      // pass 2: phi, escape test, removal
      long long rm = 0, rv0 = 0, rv1 = 0, rv2 = 0;
      int nrem = 0, nband = 0;
      for (int k = 0; k < ipt; ++k) {
        const int p = p0 + k;
        if (p < n_mem) {
          const int q = sw(p, mask);
          const float m = mm[q];
          if (!signbit(m)) {
            const float ri = rinv_of(rr[q], P.r_soft_f);
            const long long mfix = fix_from_float(m, s_m);
            const long long rfix = fix_from_float(m * ri, s_r);
            const float inner = float_from_fix(tm, s_m) * ri;
            const float outer = float_from_fix(T_tot - tr, s_r);
            const float phi = -P.Gf * (inner + outer);
            const float ux = wx[q] - vb0, uy = wy[q] - vb1, uz = wz[q] - vb2;
            const float u2 = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
            const float two_phi = -2.0f * phi;
            if (fabsf(u2 - two_phi) < P.band_f * two_phi) ++nband;
            if (u2 > two_phi) {
              mm[q] = -m;
              ++nrem;
              const int j = (int)jj[q];
              const long long slot = H.offset + j;
              const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
              float v[3];
              load_velocity<CT>(L.p, pi, v);
              rm += mfix;
              rv0 += fix_from_float(__fmul_rn(m, v[0]), s_v);
              rv1 += fix_from_float(__fmul_rn(m, v[1]), s_v);
              rv2 += fix_from_float(__fmul_rn(m, v[2]), s_v);
              if (L.out.removed_iter) L.out.removed_iter[slot] = n_iter;
            }
            tm += mfix;
            tr += rfix;
          }
        }
      }
      nrem = __reduce_add_sync(FULL_MASK, nrem);
      nband = __reduce_add_sync(FULL_MASK, nband);
      if (__any_sync(FULL_MASK, rm != 0 || rv0 != 0 || rv1 != 0 || rv2 != 0)) {
        rm = warp_sum(rm); rv0 = warp_sum(rv0); rv1 = warp_sum(rv1); rv2 = warp_sum(rv2);
        if (lane == 0) {
          atomicAdd((unsigned long long*)&S.rem[0], (unsigned long long)rm);
          atomicAdd((unsigned long long*)&S.rem[1], (unsigned long long)rv0);
          atomicAdd((unsigned long long*)&S.rem[2], (unsigned long long)rv1);
          atomicAdd((unsigned long long*)&S.rem[3], (unsigned long long)rv2);
        }
      }
      if (lane == 0 && (nrem | nband)) {
        atomicAdd(&S.removed, nrem);
        atomicAdd(&S.band, nband);
      }
      __syncthreads();
      const int removed = S.removed;
      n_band += S.band;
      if (tid == 0) {
        S.mv[0] -= S.rem[1];
        S.mv[1] -= S.rem[2];
        S.mv[2] -= S.rem[3];
      }
      __syncthreads();
      n_alive -= removed;
      if (removed == 0) { converged = true; break; }
    }
    if (n_alive == 0) status |= AHF_HALO_EMPTY;
    else if (!converged) status |= AHF_HALO_NOT_CONVERGED;

    // ---- emit: bound list, phi, compacted (r, inclusive M) for the virial search ----
    float* rc = wx;                       // reuse: w is no longer needed
    long long* mc = (long long*)ex1;      // ex1 and ex2 are contiguous
    {
      long long tm = 0, tr = 0, tc = 0;
      for (int k = 0; k < ipt; ++k) {
        const int p = p0 + k;
        if (p < n_mem) {
          const int q = sw(p, mask);
          const float m = mm[q];
          if (!signbit(m)) {
            tm += fix_from_float(m, s_m);
            tr += fix_from_float(m * rinv_of(rr[q], P.r_soft_f), s_r);
            tc += 1;
          }
        }
      }
      long long M_tot, T_tot, C_tot;
      block_exclusive_scan3<NT>(tm, tr, tc, S, M_tot, T_tot, C_tot);
      for (int k = 0; k < ipt; ++k) {
        const int p = p0 + k;
        if (p < n_mem) {
          const int q = sw(p, mask);
          const float m = mm[q];
          if (!signbit(m)) {
            const float r = rr[q];
            const float ri = rinv_of(r, P.r_soft_f);
            const long long mfix = fix_from_float(m, s_m);
            const float inner = float_from_fix(tm, s_m) * ri;
            const float outer = float_from_fix(T_tot - tr, s_r);
            const float phi = -P.Gf * (inner + outer);
            const int j = (int)jj[q];
            const long long slot = H.offset + j;
            const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
            const long long dst = H.offset + tc;
            L.out.bound_idx[dst] = pi;
            if (L.out.phi) ((float*)L.out.phi)[dst] = phi;
            if (L.out.removed_iter) L.out.removed_iter[slot] = 0;
            const int kq = sw((int)tc, mask);
            rc[kq] = r;
            mc[kq] = tm + mfix;
            tm += mfix;
            tr += fix_from_float(m * ri, s_r);
            tc += 1;
          }
        }
      }
      if (tid == 0) S.k_first = 0x7fffffff;
      __syncthreads();
      // virial: first k with M_k < delta_rho 4pi/3 r_{k+1}^3 (r_{N+1} = inf)
      const int nb = (int)C_tot;
      int kf = 0x7fffffff;
      for (int k = 0; k < ipt; ++k) {
        const int kk = p0 + k;
        if (kk < nb) {
          bool cross = true;
          if (kk + 1 < nb) {
            const float rn = rc[sw(kk + 1, mask)];
            const long long mk = mc[sw(kk, mask)];
            const float lhs = float_from_fix(mk, s_m);
            const float rhs = P.crit_f * rn * rn * rn;
            if (lhs < rhs * (1.0f - 1e-5f)) cross = true;
            else if (lhs > rhs * (1.0f + 1e-5f)) cross = false;
            else {
              const double rd = (double)rn;
              cross = double_from_fix(mk, s_m) < P.crit * rd * rd * rd;
            }
          }
          if (cross) { kf = kk; break; }
        }
      }
      kf = __reduce_min_sync(FULL_MASK, (unsigned)kf);
      if (lane == 0 && kf != 0x7fffffff) atomicMin(&S.k_first, kf);
      __syncthreads();
      if (tid == 0) {
        ahf_result R;
        R.n_bound = nb;
        R.n_member = n_mem;
        R.part_iter = part_iter;
        R.n_band = n_band;
        R.n_iter = n_iter;
        R.k_vir = -1;
        R.m_vir = 0.0;
        R.r_vir = 0.0;
        if (nb > 0) {
          const int k = S.k_first;
          const double mk = double_from_fix(mc[sw(k, mask)], s_m);
          const double rk = (double)rc[sw(k, mask)];
          if (k == nb - 1) status |= AHF_HALO_RVIR_BEYOND_EDGE;
          if (mk < P.crit * rk * rk * rk) {
            status |= AHF_HALO_RVIR_NONE;
          } else {
            R.k_vir = k;
            R.m_vir = mk;
            R.r_vir = cbrt(mk / P.crit);
          }
          const double mt = double_from_fix(M_tot, s_m);
          for (int c = 0; c < 3; ++c) R.vbulk[c] = double_from_fix(S.mv[c], s_v) / mt;
        } else {
          R.vbulk[0] = R.vbulk[1] = R.vbulk[2] = 0.0;
        }
        R.status = status;
        L.out.res[H.index] = R;
      }
    }
    __syncthreads();
  }
}

// variant table: (threads, capacity)
template <int NT, int CAP>
constexpr size_t dyn_bytes() {
  return (size_t)CAP * 24 + (size_t)(NT / 32) * 256 * 2;
}

template <int NT, int CAP, int CT>
cudaError_t launch_variant(const OnchipLaunch& L, int grid, cudaStream_t s) {
  auto k = onchip_kernel<NT, CAP, CT>;
  constexpr size_t smem = dyn_bytes<NT, CAP>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, smem, s>>>(L);
  return cudaGetLastError();
}

template <int NT, int CAP>
int max_grid_variant(int device) {
  int per_sm = 0, sms = 0;
  constexpr size_t smem = dyn_bytes<NT, CAP>();
  cudaFuncSetAttribute(onchip_kernel<NT, CAP, AHF_COORD_F32_REL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onchip_kernel<NT, CAP, AHF_COORD_F32_REL>, NT,
                                                    smem) != cudaSuccess)
    per_sm = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return (per_sm > 0 ? per_sm : 1) * sms;
}

}  // namespace

// Variants: 0 = 128 threads / 1024 slots, 1 = 256 / 4096, 2 = 512 / 8192.
int onchip_capacity(int variant) {
  switch (variant) {
    case 0: return 1024;
    case 1: return 4096;
    case 2: return 8192;
    default: return 0;
  }
}

int onchip_max_grid(int variant, int device) {
  switch (variant) {
    case 0: return max_grid_variant<128, 1024>(device);
    case 1: return max_grid_variant<256, 4096>(device);
    case 2: return max_grid_variant<512, 8192>(device);
    default: return 0;
  }
}

cudaError_t launch_onchip(const OnchipLaunch& L, int variant, int grid, cudaStream_t s) {
  const bool f64 = L.p.coord_type == AHF_COORD_F64;
  switch (variant) {
    case 0: return f64 ? launch_variant<128, 1024, AHF_COORD_F64>(L, grid, s)
                       : launch_variant<128, 1024, AHF_COORD_F32_REL>(L, grid, s);
    case 1: return f64 ? launch_variant<256, 4096, AHF_COORD_F64>(L, grid, s)
                       : launch_variant<256, 4096, AHF_COORD_F32_REL>(L, grid, s);
    case 2: return f64 ? launch_variant<512, 8192, AHF_COORD_F64>(L, grid, s)
                       : launch_variant<512, 8192, AHF_COORD_F32_REL>(L, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ahf
