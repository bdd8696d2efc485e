// On-chip classes: a halo unbound entirely in shared memory, by one CTA or
// by a thread-block cluster of CS CTAs sharing their shared memory (DSMEM).
//
// Per halo (Sect. 2.1 and Appendix A):
//   gather   candidates -> (radius key, candidate position), FP64-accurate
//            recentring and sphere test, exponent maxima for the exact sums;
//            each member's offset, mass and velocity to its 32-byte record
//   sort     stable LSD radix sort of the keys, once: the centre is fixed and
//            particles only leave, so the survivors of every later iteration
//            stay in radial order.  One CTA ranks 5-bit digits by counting
//            (count_sort); a cluster ranks 8-bit digits by lane matching, each
//            CTA holding a contiguous chunk of the order, the scatter writing
//            into the owner CTA's shared memory.
//   fill     sorted SoA from the records: radius, mass, w = v + H d; exact
//            sum m v
//   iterate  scan of the exact M(<r) and sum m/r prefixes ->
//            phi_i = -G [M(<r_i)/r_i + sum_{j>=i} m_j/r_j], escape test
//            |w - v_bulk|^2 > 2|phi|, removal of every unbound particle, until
//            an iteration removes nothing.  Each thread keeps the exact sums
//            of its own particles and subtracts what it removes, so one pass
//            over the particles per iteration suffices.
//   emit     bound list (particle index, phi) in radial order, virial crossing
//            of the final set (Sect. 2.1, Eqs. 1-2), result record
//
// CTAs (clusters) are persistent: each pulls the next halo from a counter over
// the class's haloes, which the host orders largest first.  Cross-CTA values
// go through a small exchange record in each CTA's shared memory, read by the
// others after a hardware cluster barrier; every CTA combines them in rank
// order, so all CTAs hold identical cluster-wide values.
#include <cooperative_groups.h>

#include <cstdint>

#include "ahf_device.cuh"

namespace cg = cooperative_groups;

namespace ahf {
namespace {

// Swizzled shared-memory position of element p for a blocked arrangement of
// ipt = mask + 1 consecutive elements per thread: conflict-free both for
// per-thread runs and for warp-striped access.
__device__ __forceinline__ int sw(int p, int mask) { return p ^ ((p >> 5) & mask); }

template <int CS>
struct Cl {
  static __device__ __forceinline__ int rank() {
    if constexpr (CS > 1) return (int)cg::this_cluster().block_rank();
    else return 0;
  }
  static __device__ __forceinline__ void sync() {
    if constexpr (CS > 1) cg::this_cluster().sync();
    else __syncthreads();
  }
  template <typename T>
  static __device__ __forceinline__ T* at(T* p, int r) {
    if constexpr (CS > 1) return cg::this_cluster().map_shared_rank(p, r);
    else return p;
  }
};

// Largest bin count a cluster forms profile rows for itself (larger requests
// use the profile kernels).
constexpr int FUSE_BINS = 128;

// Values a CTA publishes to the other CTAs of its cluster.
struct Xchg {
  int halo;
  uint32_t g_or, g_and, g_mxm, g_mxr, g_mxv;
  int g_nmem;
  uint32_t cnt[256];            // radix pass: digit counts of this CTA
  long long mv[3];              // fill: partial sum m v
  // iteration exchange, two alternating copies: scan totals of this CTA
  // (M, sum m/r, count) and its removals of the previous iteration (m,
  // m v (3), count, band count)
  long long xt[2][3];
  long long xr[2][4];
  int xn[2], xb[2];
  float first_r;                // emit: first compacted radius of this CTA
  int nb_loc;                   // emit: bound particles held by this CTA
  int kf;                       // emit: first local virial crossing (global index)
  // fused profile rows: r_vir from the owner CTA, last radius, and this CTA's
  // bound count and inclusive mass at every bin edge
  double rvir;
  int has_rvir;
  float last_r;
  int pc[FUSE_BINS + 1];
  long long pm[FUSE_BINS + 1];
};

template <int NT>
struct Smem {
  static constexpr int NW = NT / 32;
  long long red[NW][4];
  long long scan_base[NW][3];
  long long tot[3];
  uint32_t or_bits, and_bits, max_m, max_mr, max_mv;
  uint32_t max_key;             // largest member key (single-CTA sort)
  int n_member;
  long long acc[4];             // block accumulators (m v or removed m, m v)
  int acc_n, acc_band;
  // one CTA's removal sums, alternating between iterations: (removed m, m v),
  // removed count, band count
  long long racc[2][4];
  int racc_n[2], racc_band[2];
  // cluster-wide values
  long long c_pre[3];           // exclusive prefix over lower ranks
  long long c_tot[3];
  long long mv[3];              // exact sum m v of the current set
  int c_removed, c_band;
  int k_first;
  float vb[3];
  double rvir;                  // emit: the record's r_vir, for the profile rows
  uint32_t dtot[256];
  uint32_t dpre[256];
};

template <int NT>
__device__ __forceinline__ void block_exclusive_scan3(long long& a, long long& b, long long& c, Smem<NT>& S) {
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
}

// The same for two values (the iterations need no count): totals in
// S.tot[0], S.tot[1].
template <int NT>
__device__ __forceinline__ void block_exclusive_scan2(long long& a, long long& b, Smem<NT>& S) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long ia = warp_inclusive_scan(a, lane);
  long long ib = warp_inclusive_scan(b, lane);
  if (lane == 31) { S.red[warp][0] = ia; S.red[warp][1] = ib; }
  __syncthreads();
  if (warp == 0) {
    long long x = lane < NW ? S.red[lane][0] : 0, y = lane < NW ? S.red[lane][1] : 0;
    long long sx = warp_inclusive_scan(x, lane), sy = warp_inclusive_scan(y, lane);
    if (lane < NW) { S.scan_base[lane][0] = sx - x; S.scan_base[lane][1] = sy - y; }
    if (lane == NW - 1) { S.tot[0] = sx; S.tot[1] = sy; }
  }
  __syncthreads();
  a = S.scan_base[warp][0] + ia - a;
  b = S.scan_base[warp][1] + ib - b;
}

// One exchange of a cluster iteration: every CTA publishes its scan totals
// of the current set and its removal sums of the previous iteration (zero
// before the first) in copy `xs`, and combines the cluster's: S.c_pre gets
// the totals over lower ranks, S.c_tot over all ranks; S.mv loses the m v
// removed, S.c_removed and S.c_band count the removed and the band.  The
// copies alternate between iterations: a CTA writes copy xs again only
// after the next exchange's barrier, which every reader of this one has
// passed after reading it.
template <int NT, int CS>
__device__ __forceinline__ void cluster_exchange(Smem<NT>& S, Xchg& X, int rank, int xs, bool first) {
  if (threadIdx.x == 0) {
    X.xt[xs][0] = S.tot[0]; X.xt[xs][1] = S.tot[1]; X.xt[xs][2] = S.tot[2];
    X.xr[xs][0] = first ? 0 : S.acc[0];
    X.xr[xs][1] = first ? 0 : S.acc[1];
    X.xr[xs][2] = first ? 0 : S.acc[2];
    X.xr[xs][3] = first ? 0 : S.acc[3];
    X.xn[xs] = first ? 0 : S.acc_n;
    X.xb[xs] = first ? 0 : S.acc_band;
  }
  Cl<CS>::sync();
  if (threadIdx.x < 3) {
    long long pre = 0, tot = 0;
#pragma unroll
    for (int r = 0; r < CS; ++r) {
      const long long v = Cl<CS>::at(&X.xt[xs][0], r)[threadIdx.x];
      if (r < rank) pre += v;
      tot += v;
    }
    S.c_pre[threadIdx.x] = pre;
    S.c_tot[threadIdx.x] = tot;
  } else if (threadIdx.x == 32) {
    long long a1 = 0, a2 = 0, a3 = 0;
    int nr = 0, nbd = 0;
#pragma unroll
    for (int r = 0; r < CS; ++r) {
      const Xchg* Y = Cl<CS>::at(&X, r);
      a1 += Y->xr[xs][1]; a2 += Y->xr[xs][2]; a3 += Y->xr[xs][3];
      nr += Y->xn[xs]; nbd += Y->xb[xs];
    }
    S.mv[0] -= a1; S.mv[1] -= a2; S.mv[2] -= a3;
    S.c_removed = nr;
    S.c_band = nbd;
  }
  __syncthreads();
}

// Stable LSD radix sort of the halo's keys, 8-bit digits, skipping the digits
// in which all keys agree.  Each CTA of the cluster holds `nloc` elements of a
// chunk of `chunk` positions, in order; the result keeps that partition, with
// element p of a CTA at sw(p, mask).  Every pass scatters (key, value) pairs
// as one 8-byte store into the owner CTA's shared memory (the two arrays of a
// buffer, kA|vA or kB|vB, hold CAP interleaved pairs between passes); a local
// pass splits the final pairs into the other buffer.  Returns 0 if the result
// is in (kA, vA), 1 if in (kB, vB) (the same in every CTA).
template <int NT, int IPT, int CS>
__device__ int cluster_radix_sort(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, uint16_t* hist, Smem<NT>& S,
                                  Xchg& X, int nloc, int chunk, uint32_t diff, int mask, int rank) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int passes[4], np = 0;
  for (int d = 0; d < 4; ++d)
    if ((diff >> (8 * d)) & 0xffu) passes[np++] = d;
  if (np == 0) {
    for (int p = threadIdx.x; p < nloc; p += NT) {
      kB[sw(p, mask)] = kA[p];
      vB[sw(p, mask)] = vA[p];
    }
    __syncthreads();
    return 1;
  }
  uint2* pA = reinterpret_cast<uint2*>(kA);     // kA|vA as interleaved pairs
  uint2* pB = reinterpret_cast<uint2*>(kB);     // kB|vB
  uint2 *pin = pA, *pout = pB;
  const int wchunk = ((nloc + NW * 32 - 1) / (NW * 32)) * 32;   // per-warp run
  const int nb = wchunk / 32;                                   // <= IPT
  for (int ip = 0; ip < np; ++ip) {
    const int shift = 8 * passes[ip];
    for (int i = threadIdx.x; i < NW * 256; i += NT) hist[i] = 0;
    __syncthreads();
    // keys are read again for the scatter (the input buffer does not change
    // during a pass): only the ranks stay in registers
    uint16_t rank_in[IPT];
#pragma unroll
    for (int b = 0; b < IPT; ++b) {
      if (b < nb) {
        const int e = warp * wchunk + b * 32 + lane;
        const bool valid = e < nloc;
        const uint32_t key = valid ? (ip == 0 ? kA[e] : pin[e].x) : 0u;   // pass 0: the gather's arrays
        const unsigned vmask = __ballot_sync(FULL_MASK, valid);
        rank_in[b] = 0;
        if (valid) {
          const uint32_t dg = (key >> shift) & 0xffu;
          const unsigned peers = __match_any_sync(vmask, dg);
          const unsigned below = peers & lanemask_lt();
          const uint16_t base = hist[warp * 256 + dg];
          rank_in[b] = (uint16_t)(base + __popc(below));
          __syncwarp(vmask);
          if (below == 0) hist[warp * 256 + dg] = (uint16_t)(base + __popc(peers));
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // this CTA's digit counts; per-warp counts become within-CTA offsets
    for (int dg = threadIdx.x; dg < 256; dg += NT) {
      uint32_t run = 0;
      for (int w = 0; w < NW; ++w) {
        const uint32_t h = hist[w * 256 + dg];
        hist[w * 256 + dg] = (uint16_t)run;
        run += h;
      }
      X.cnt[dg] = run;
    }
    Cl<CS>::sync();
    // cluster: digit totals, and counts of this digit in lower-ranked CTAs
    for (int dg = threadIdx.x; dg < 256; dg += NT) {
      uint32_t tot = 0, pre = 0;
      for (int r = 0; r < CS; ++r) {
        const uint32_t v = Cl<CS>::at(X.cnt, r)[dg];
        if (r < rank) pre += v;
        tot += v;
      }
      S.dtot[dg] = tot;
      S.dpre[dg] = pre;
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t loc[8], s = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { loc[i] = S.dtot[lane * 8 + i]; s += loc[i]; }
      const uint32_t inc = warp_inclusive_scan(s, lane);
      uint32_t run = inc - s;
#pragma unroll
      for (int i = 0; i < 8; ++i) { S.dtot[lane * 8 + i] = run + S.dpre[lane * 8 + i]; run += loc[i]; }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < IPT; ++b) {
      if (b < nb) {
        const int e = warp * wchunk + b * 32 + lane;
        if (e < nloc) {
          const uint2 kv = ip == 0 ? make_uint2(kA[e], vA[e]) : pin[e];
          const uint32_t dg = (kv.x >> shift) & 0xffu;
          const int g = (int)S.dtot[dg] + (int)hist[warp * 256 + dg] + (int)rank_in[b];
          const int q = g / chunk;
          Cl<CS>::at(pout, q)[g - q * chunk] = kv;
        }
      }
    }
    Cl<CS>::sync();
    uint2* t = pin;
    pin = pout;
    pout = t;
  }
  // split this CTA's sorted pairs into the other buffer, swizzled
  uint32_t* ko = reinterpret_cast<uint32_t*>(pout);
  uint32_t* vo = ko + IPT * NT;
  for (int p = threadIdx.x; p < nloc; p += NT) {
    const uint2 x = pin[p];
    ko[sw(p, mask)] = x.x;
    vo[sw(p, mask)] = x.y;
  }
  __syncthreads();
  return pout == pA ? 0 : 1;
}

template <int NT, int CS>
constexpr int min_blocks() { return CS > 1 ? 1 : (NT <= 128 ? 6 : (NT <= 256 ? 2 : 1)); }

template <int NT, int CAP, int CT, int CS>
__global__ void __launch_bounds__(NT, (min_blocks<NT, CS>())) unbind_kernel(OnchipLaunch L) {
  constexpr int IPT = CAP / NT;
  static_assert(IPT * NT == CAP && IPT <= 32 && (IPT & (IPT - 1)) == 0, "bad tile");
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Smem<NT> S;
  __shared__ Xchg X;
  uint32_t* kA = (uint32_t*)dyn;
  uint32_t* vA = kA + CAP;
  uint32_t* kB = vA + CAP;
  uint32_t* vB = kB + CAP;
  float* ex1 = (float*)(vB + CAP);
  float* ex2 = ex1 + CAP;
  uint16_t* hist = (uint16_t*)(ex2 + CAP);

  const int tid = threadIdx.x, lane = tid & 31;
  const int rank = Cl<CS>::rank();
  const ParamsDev& P = L.prm;

  for (;;) {
    if (rank == 0 && tid == 0) X.halo = atomicAdd(L.queue, 1);
    Cl<CS>::sync();
    const int hq = *Cl<CS>::at(&X.halo, 0);
    Cl<CS>::sync();
    if (hq >= L.n_halos) break;
    const HaloDev& H = L.halos[hq];
    if (tid == 0 && rank == 0) trace_mark(L.trace, H.index, 0);
    const int n_cand = (int)H.count;
    const int chunk = n_cand > 0 ? (n_cand + CS - 1) / CS : 1;
    if (chunk > CAP) {    // the scheduler never does this; report, do not overrun
      if (tid == 0 && rank == 0) atomicOr(L.out.err, ERR_CAPACITY);
      continue;
    }
    const int lo = rank * chunk;
    const int nloc = max(0, min(n_cand - lo, chunk));
    int ipt = 1;
    while (ipt * NT < chunk) ipt <<= 1;
    const int mask = ipt - 1;
    prefetch_candidates<CT>(L.p, L.out.member_idx, H.offset + lo, H.offset + lo + nloc, tid);
    if (tid == 0) {
      S.or_bits = 0u; S.and_bits = 0xffffffffu;
      S.max_m = 0u; S.max_mr = 0u; S.max_mv = 0u;
      S.max_key = 0u;
      S.n_member = 0;
      S.acc[0] = S.acc[1] = S.acc[2] = S.acc[3] = 0;
      S.acc_n = 0; S.acc_band = 0;
    }
    __syncthreads();

    // ---- gather: key = radius bits of members, candidate position as value ----
    {
      uint32_t orb = 0u, andb = 0xffffffffu, mxm = 0u, mxr = 0u, mxv = 0u, kmx = 0u;
      int nmem = 0;
      for (int i = tid; i < nloc; i += NT) {
        const int j = lo + i;
        const long long slot = H.offset + j;
        long long pi = slot;
        bool ok = true;
        if (L.out.member_idx) {
          pi = L.out.member_idx[slot];
          if (pi < 0 || pi >= L.p.n) { ok = false; atomicOr(L.out.err, ERR_BAD_INDEX); }
        }
        uint32_t key = KEY_NONMEMBER;
        if (ok) {
          Cand<CT> c;
          load_cand<CT>(L.p, pi, c);
          long long f[3];
          float df[3];
          cand_offset<CT>(c, H, df, f);
          if (cand_member<CT>(c, H, df, f)) {
            const float r = radius_of(df);
            key = __float_as_uint(r);
            const float m = cand_mass<CT>(L.p, c);
            float v[3];
            cand_velocity<CT>(c, v);
            if (L.rec) put_record(L.rec + 2 * (H.gbase + j), df, m, v);
            mxm = max(mxm, __float_as_uint(fabsf(m)));
            mxr = max(mxr, __float_as_uint(fabsf(m * rinv_of(r, P.r_soft_f))));
#pragma unroll
            for (int k = 0; k < 3; ++k) mxv = max(mxv, __float_as_uint(fabsf(__fmul_rn(m, v[k]))));
            ++nmem;
          }
        }
        // members start bound (removal overwrites with its iteration)
        if (L.out.removed_iter) L.out.removed_iter[slot] = key == KEY_NONMEMBER ? -1 : 0;
        // one CTA sorts runs of ipt consecutive positions (swizzled), a
        // cluster contiguous chunks; the single-CTA sort's key range is
        // the members' (non-members get a key just above it)
        const int wpos = CS == 1 ? sw(i, mask) : i;
        kA[wpos] = key;
        vA[wpos] = (uint32_t)j;
        if (CS > 1 || key != KEY_NONMEMBER) {
          orb |= key;
          andb &= key;
          kmx = max(kmx, key);
        }
      }
      orb = __reduce_or_sync(FULL_MASK, orb);
      andb = __reduce_and_sync(FULL_MASK, andb);
      mxm = __reduce_max_sync(FULL_MASK, mxm);
      mxr = __reduce_max_sync(FULL_MASK, mxr);
      mxv = __reduce_max_sync(FULL_MASK, mxv);
      nmem = __reduce_add_sync(FULL_MASK, nmem);
      if constexpr (CS == 1) kmx = __reduce_max_sync(FULL_MASK, kmx);
      if (lane == 0) {
        if constexpr (CS == 1) atomicMax(&S.max_key, kmx);
        atomicOr(&S.or_bits, orb);
        atomicAnd(&S.and_bits, andb);
        atomicMax(&S.max_m, mxm);
        atomicMax(&S.max_mr, mxr);
        atomicMax(&S.max_mv, mxv);
        atomicAdd(&S.n_member, nmem);
      }
    }
    __syncthreads();
    if constexpr (CS > 1) {
      if (tid == 0) {
        X.g_or = S.or_bits; X.g_and = S.and_bits; X.g_mxm = S.max_m; X.g_mxr = S.max_mr; X.g_mxv = S.max_mv;
        X.g_nmem = S.n_member;
      }
      Cl<CS>::sync();
      if (tid == 0) {
        uint32_t o = 0u, a = 0xffffffffu, m1 = 0u, m2 = 0u, m3 = 0u;
        int nm = 0;
        for (int r = 0; r < CS; ++r) {
          const Xchg* Y = Cl<CS>::at(&X, r);
          o |= Y->g_or; a &= Y->g_and;
          m1 = max(m1, Y->g_mxm); m2 = max(m2, Y->g_mxr); m3 = max(m3, Y->g_mxv);
          nm += Y->g_nmem;
        }
        S.or_bits = o; S.and_bits = a; S.max_m = m1; S.max_mr = m2; S.max_mv = m3; S.n_member = nm;
      }
      __syncthreads();
    }
    const int n_mem = S.n_member;                        // members of the halo
    const int nmem_loc = max(0, min(n_mem - lo, nloc));  // held by this CTA after the sort
    const int s_m = fix_scale(float_exponent_of_bits(S.max_m), n_mem);
    const int s_r = fix_scale(float_exponent_of_bits(S.max_mr), n_mem);
    const int s_v = fix_scale(float_exponent_of_bits(S.max_mv), n_mem);
    const bool unim = L.p.m == nullptr;                  // every particle has mass m0
    const long long m0fix = fix_from_float(L.p.m0f, s_m);
    // 2^-s of the mass and m/r sums as floats (0 when not normal): each
    // exact sum's float value is then one multiply, the bits of float_from_fix
    const float sc_m = pow2_neg(s_m), sc_r = pow2_neg(s_r);

    if (tid == 0 && rank == 0) trace_mark(L.trace, H.index, 1);
    // ---- radial sort (once) ----
    int which;
    if constexpr (CS == 1) {
      uint32_t diff = 0u, sub = 0u;
      if (n_mem > 0) {
        diff = S.or_bits ^ S.and_bits;
        if (n_mem < n_cand) {
          sub = S.max_key + 1u;
          diff = (S.or_bits | sub) ^ (S.and_bits & sub);
        }
      }
      which = count_sort<NT, IPT>(kA, vA, kB, vB, reinterpret_cast<uint32_t*>(hist),
                                  reinterpret_cast<uint32_t*>(&S.red[0][0]), nloc, mask, diff, sub, tid);
    } else {
      which = cluster_radix_sort<NT, IPT, CS>(kA, vA, kB, vB, hist, S, X, nloc, chunk, S.or_bits ^ S.and_bits,
                                              mask, rank);
    }
    if (tid == 0 && rank == 0) trace_mark(L.trace, H.index, 2);
    float* rr = (float*)(which ? kB : kA);         // radius, sorted, swizzled
    uint32_t* jj = which ? vB : vA;                // candidate position
    float* mm = (float*)(which ? kA : kB);         // mass; sign bit = removed
    float* wx = (float*)(which ? vA : vB);
    float* wy = ex1;
    float* wz = ex2;

    // ---- fill: m and w = v + H d in the radial order, and the exact sum m v
    // of the members (the sorted candidates re-read from the store, mostly L2)
    const int p0 = tid * ipt;
    {
      long long smv[3] = {0, 0, 0};
      for (int p = tid; p < nmem_loc; p += NT) {
        const int q = sw(p, mask);
        const int j = (int)jj[q];
        float dfl[3], v[3], m;
        if (L.rec) {
          get_record(L.rec + 2 * (H.gbase + j), dfl, m, v);
        } else {
          const long long slot = H.offset + j;
          const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
          long long f[3];
          offset_of<CT>(L.p, pi, H, dfl, f);
          load_velocity<CT>(L.p, pi, v);
          m = load_mass<CT>(L.p, pi);
        }
        // with a uniform mass the slot holds 1 / max(r, r_soft) instead (the
        // mass is m0): the reciprocal is formed once, not every iteration
        mm[q] = unim ? rinv_of(rr[q], P.r_soft_f) : m;
        wx[q] = fmaf(P.Hf, dfl[0], v[0]);
        wy[q] = fmaf(P.Hf, dfl[1], v[1]);
        wz[q] = fmaf(P.Hf, dfl[2], v[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) smv[k] += fix_from_float(__fmul_rn(m, v[k]), s_v);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const long long t = warp_sum(smv[k]);
        if (lane == 0 && t != 0) atomicAdd((unsigned long long*)&S.acc[k], (unsigned long long)t);
      }
    }
    __syncthreads();
    if constexpr (CS > 1) {
      if (tid == 0) { X.mv[0] = S.acc[0]; X.mv[1] = S.acc[1]; X.mv[2] = S.acc[2]; }
      Cl<CS>::sync();
      if (tid < 3) {
        long long t = 0;
        for (int r = 0; r < CS; ++r) t += Cl<CS>::at(&X.mv[0], r)[tid];
        S.mv[tid] = t;
      }
    } else {
      if (tid < 3) S.mv[tid] = S.acc[tid];
    }
    __syncthreads();

    if (tid == 0 && rank == 0) trace_mark(L.trace, H.index, 3);
    // per-thread exact sums of m, m/r and the alive count over its run
    long long tm_own = 0, tr_own = 0, tc_own = 0;
    for (int k = 0; k < ipt; ++k) {
      const int p = p0 + k;
      if (p < nmem_loc) {
        const int q = sw(p, mask);
        const float mq = mm[q];
        const float m = unim ? L.p.m0f : mq;
        const float ri = unim ? mq : rinv_of(rr[q], P.r_soft_f);
        tm_own += (unim ? m0fix : fix_from_float(m, s_m));
        tr_own += fix_from_float(m * ri, s_r);
        tc_own += 1;
      }
    }

    // ---- iterate (Appendix A) ----
    int n_iter = 0, status = 0;
    long long part_iter = 0, n_band = 0;
    int n_alive = n_mem;
    bool converged = false;
    // one CTA: every thread keeps the exact sum m v and forms v_bulk itself
    // (the same bits in every thread), and the removal sums alternate
    // between two buffers, so an iteration takes three barriers
    long long mvl[3] = {S.mv[0], S.mv[1], S.mv[2]};
    float vbl[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (CS == 1) {
      if (tid == 0)
        for (int bsel = 0; bsel < 2; ++bsel) {
          S.racc[bsel][0] = S.racc[bsel][1] = S.racc[bsel][2] = S.racc[bsel][3] = 0;
          S.racc_n[bsel] = 0;
          S.racc_band[bsel] = 0;
        }
    }
    // a cluster: one exchange per iteration (cluster_exchange) carries the
    // scan totals of the current set and the previous iteration's removals;
    // the last one, of the final set, also serves the emit
    long long e_tm = 0, e_tr = 0, e_tc = 0;   // the emit's prefixes (cluster)
    int xs = 0;
    for (;;) {
      long long tm = tm_own, tr = tr_own;
      long long T_tot;
      int bsel = 0;
      if constexpr (CS == 1) {
        if (!(n_alive > 0 && n_iter < P.max_iter)) break;
        ++n_iter;
        part_iter += n_alive;
        bsel = n_iter & 1;
        block_exclusive_scan2<NT>(tm, tr, S);
        T_tot = S.tot[1];
        // v_bulk = sum m v / sum m of the current set, from the exact sums
        // (with AHF_VAR_VBULK_INITIAL the first iteration's value is kept)
        if (n_iter == 1 || !P.vbulk_initial) {
          const float mt = float_from_fix(S.tot[0], s_m);
          vbl[0] = float_from_fix(mvl[0], s_v) / mt;
          vbl[1] = float_from_fix(mvl[1], s_v) / mt;
          vbl[2] = float_from_fix(mvl[2], s_v) / mt;
        }
        if (tid == 0) {                  // the next iteration's buffer: its readers are past the scan
          S.racc[bsel ^ 1][0] = S.racc[bsel ^ 1][1] = S.racc[bsel ^ 1][2] = S.racc[bsel ^ 1][3] = 0;
          S.racc_n[bsel ^ 1] = 0;
          S.racc_band[bsel ^ 1] = 0;
        }
      } else {
        long long tc = tc_own;
        block_exclusive_scan3<NT>(tm, tr, tc, S);
        cluster_exchange<NT, CS>(S, X, rank, xs, n_iter == 0);
        xs ^= 1;
        bool stop = false;
        if (n_iter > 0) {                // the previous iteration's removals
          const int removed = S.c_removed;
          n_band += S.c_band;
          n_alive -= removed;
          if (removed == 0) {
            converged = true;
            stop = true;
          }
        }
        if (stop || !(n_alive > 0 && n_iter < P.max_iter)) {
          e_tm = tm;
          e_tr = tr;
          e_tc = tc;
          break;
        }
        ++n_iter;
        part_iter += n_alive;
        if (tid == 0) {
          if (n_iter == 1 || !P.vbulk_initial) {
            const float mt = float_from_fix(S.c_tot[0], s_m);
            S.vb[0] = float_from_fix(S.mv[0], s_v) / mt;
            S.vb[1] = float_from_fix(S.mv[1], s_v) / mt;
            S.vb[2] = float_from_fix(S.mv[2], s_v) / mt;
          }
          S.acc[0] = S.acc[1] = S.acc[2] = S.acc[3] = 0;
          S.acc_n = 0;
          S.acc_band = 0;
        }
        __syncthreads();
        tm += S.c_pre[0];
        tr += S.c_pre[1];
        T_tot = S.c_tot[1];
        vbl[0] = S.vb[0];
        vbl[1] = S.vb[1];
        vbl[2] = S.vb[2];
      }
      const float vb0 = vbl[0], vb1 = vbl[1], vb2 = vbl[2];
      long long rm = 0, rq = 0, rv0 = 0, rv1 = 0, rv2 = 0;
      int nrem = 0, nband = 0;
      uint32_t rmask = 0;                 // this thread's removals (bit k: position p0 + k)
      // no branch per member: a slot past the members or removed earlier
      // adds nothing and is not tested (every slot of the run is within the
      // arrays), so the loop's members can overlap
      if (p0 < nmem_loc) {
#pragma unroll 4
        for (int k = 0; k < ipt; ++k) {
          const int p = p0 + k;
          const int q = sw(p, mask);
          const float mq = mm[q];
          const bool alive = p < nmem_loc && !signbit(mq);
          const float m = unim ? L.p.m0f : mq;
          const float ri = unim ? mq : rinv_of(rr[q], P.r_soft_f);
          const long long mfix = alive ? (unim ? m0fix : fix_from_float(m, s_m)) : 0ll;
          const long long rfix = alive ? fix_from_float(m * ri, s_r) : 0ll;
          const float phi = phi_of(fix_to_float_fast(tm, s_m, sc_m), ri, fix_to_float_fast(T_tot - tr, s_r, sc_r),
                                   P.Gf);
          const float ux = wx[q] - vb0, uy = wy[q] - vb1, uz = wz[q] - vb2;
          const float u2 = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
          const float two_phi = -2.0f * phi;
          nband += (alive && fabsf(u2 - two_phi) < P.band_f * two_phi) ? 1 : 0;
          if (alive && u2 > two_phi) {
            mm[q] = -mq;
            rmask |= 1u << k;
            rm += mfix;
            rq += rfix;
          }
          tm += mfix;
          tr += rfix;
        }
      }
      // the removed: exact m v from the stored velocity, and their record
      for (uint32_t b = rmask; b; b &= b - 1) {
        const int k = __ffs(b) - 1;
        const int q = sw(p0 + k, mask);
        const float m = unim ? L.p.m0f : -mm[q];
        const int j = (int)jj[q];
        const long long slot = H.offset + j;
        float v[3];
        if (L.rec) get_velocity_record(L.rec + 2 * (H.gbase + j), v);
        else load_velocity<CT>(L.p, L.out.member_idx ? L.out.member_idx[slot] : slot, v);
        rv0 += fix_from_float(__fmul_rn(m, v[0]), s_v);
        rv1 += fix_from_float(__fmul_rn(m, v[1]), s_v);
        rv2 += fix_from_float(__fmul_rn(m, v[2]), s_v);
        if (L.out.removed_iter) L.out.removed_iter[slot] = n_iter;
        ++nrem;
      }
      tm_own -= rm;
      tr_own -= rq;
      tc_own -= nrem;
      nrem = __reduce_add_sync(FULL_MASK, nrem);
      nband = __reduce_add_sync(FULL_MASK, nband);
      long long* acc = CS == 1 ? S.racc[bsel] : S.acc;
      int* acc_n = CS == 1 ? &S.racc_n[bsel] : &S.acc_n;
      int* acc_band = CS == 1 ? &S.racc_band[bsel] : &S.acc_band;
      if (nrem) {
        rm = warp_sum(rm); rv0 = warp_sum(rv0); rv1 = warp_sum(rv1); rv2 = warp_sum(rv2);
        if (lane == 0) {
          atomicAdd((unsigned long long*)&acc[0], (unsigned long long)rm);
          atomicAdd((unsigned long long*)&acc[1], (unsigned long long)rv0);
          atomicAdd((unsigned long long*)&acc[2], (unsigned long long)rv1);
          atomicAdd((unsigned long long*)&acc[3], (unsigned long long)rv2);
        }
      }
      if (lane == 0 && (nrem | nband)) {
        atomicAdd(acc_n, nrem);
        atomicAdd(acc_band, nband);
      }
      __syncthreads();
      if constexpr (CS == 1) {
        const int removed = *acc_n;
        n_band += *acc_band;
        mvl[0] -= acc[1];
        mvl[1] -= acc[2];
        mvl[2] -= acc[3];
        n_alive -= removed;
        if (removed == 0) { converged = true; break; }
      }
      // a cluster: this iteration's removal sums go out with the next exchange
    }
    if (n_alive == 0) status |= AHF_HALO_EMPTY;
    else if (!converged) status |= AHF_HALO_NOT_CONVERGED;
    if constexpr (CS == 1) {
      if (tid == 0) {                    // for the record (the emit's scan barriers order it)
        S.mv[0] = mvl[0];
        S.mv[1] = mvl[1];
        S.mv[2] = mvl[2];
      }
    }

    if (tid == 0 && rank == 0) trace_mark(L.trace, H.index, 4);
    // ---- emit: bound list, phi, compacted (r, inclusive M) for the virial search ----
    float* rc = wx;                       // reuse: w is no longer needed
    long long* mc = (long long*)ex1;      // ex1 and ex2 are contiguous
    {
      long long tm = tm_own, tr = tr_own, tc = tc_own;
      if constexpr (CS == 1) {
        block_exclusive_scan3<NT>(tm, tr, tc, S);
        if (tid < 3) {
          S.c_pre[tid] = 0;
          S.c_tot[tid] = S.tot[tid];
        }
        __syncthreads();
      } else {                            // the last exchange was of the final set
        tm = e_tm;
        tr = e_tr;
        tc = e_tc;
      }
      const long long C_pre = S.c_pre[2];
      const long long C_loc = S.tot[2];
      const long long T_tot = S.c_tot[1];
      const long long nb = S.c_tot[2];
      tm += S.c_pre[0];
      tr += S.c_pre[1];
      long long tl = tc;                  // local rank of the thread's first bound particle
      for (int k = 0; k < ipt; ++k) {
        const int p = p0 + k;
        if (p < nmem_loc) {
          const int q = sw(p, mask);
          const float mq = mm[q];
          if (!signbit(mq)) {
            const float r = rr[q];
            const float m = unim ? L.p.m0f : mq;
            const float ri = unim ? mq : rinv_of(r, P.r_soft_f);
            const long long mfix = (unim ? m0fix : fix_from_float(m, s_m));
            const float phi = phi_of(fix_to_float_fast(tm, s_m, sc_m), ri, fix_to_float_fast(T_tot - tr, s_r, sc_r),
                                     P.Gf);
            const int j = (int)jj[q];
            const long long slot = H.offset + j;
            const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
            const long long dst = H.offset + C_pre + tl;
            L.out.bound_idx[dst] = pi;
            if (L.out.phi) ((float*)L.out.phi)[dst] = phi;
            const int kq = sw((int)tl, mask);
            rc[kq] = r;
            mc[kq] = tm + mfix;
            tm += mfix;
            tr += fix_from_float(m * ri, s_r);
            tl += 1;
          }
        }
      }
      if (tid == 0) S.k_first = 0x7fffffff;
      __syncthreads();
      float r_after = __int_as_float(0x7f800000);   // +inf: radius of the next bound particle
      if constexpr (CS > 1) {
        if (tid == 0) {
          X.nb_loc = (int)C_loc;
          X.first_r = C_loc > 0 ? rc[sw(0, mask)] : 0.0f;
        }
        Cl<CS>::sync();
        for (int r2 = rank + 1; r2 < CS; ++r2) {
          const Xchg* Y = Cl<CS>::at(&X, r2);
          if (Y->nb_loc > 0) { r_after = Y->first_r; break; }
        }
      }
      // virial: first k with M_k < delta_rho 4pi/3 r_{k+1}^3 (r_{N+1} = inf)
      int kf = 0x7fffffff;
      for (int k = 0; k < ipt; ++k) {
        const int kk = p0 + k;
        if (kk < C_loc) {
          const float rn = kk + 1 < C_loc ? rc[sw(kk + 1, mask)] : r_after;
          bool cross = true;
          if (!isinf(rn)) {
            const long long mk = mc[sw(kk, mask)];
            const float lhs = fix_to_float_fast(mk, s_m, sc_m);
            const float rhs = P.crit_f * rn * rn * rn;
            if (lhs < rhs * (1.0f - 1e-5f)) cross = true;
            else if (lhs > rhs * (1.0f + 1e-5f)) cross = false;
            else {
              const double rd = (double)rn;
              cross = double_from_fix(mk, s_m) < P.crit * rd * rd * rd;
            }
          }
          if (cross) { kf = (int)(C_pre + kk); break; }
        }
      }
      kf = (int)__reduce_min_sync(FULL_MASK, (unsigned)kf);
      if (lane == 0 && kf != 0x7fffffff) atomicMin(&S.k_first, kf);
      __syncthreads();
      if constexpr (CS > 1) {
        if (tid == 0) X.kf = S.k_first;
        Cl<CS>::sync();
        if (tid == 0) {
          int k = 0x7fffffff;
          for (int r2 = 0; r2 < CS; ++r2) k = min(k, Cl<CS>::at(&X, r2)->kf);
          S.k_first = k;
        }
        __syncthreads();
      }
      // the CTA holding the crossing particle writes the record
      const int k = S.k_first;
      const bool owner = nb > 0 ? (k >= C_pre && k < C_pre + C_loc) : rank == 0;
      if (owner) {
        // the record, its FP64 parts spread over the first thread of four
        // warps (one per SM sub-partition): the virial pair, and one bulk
        // velocity component each
        ahf_result* R = L.out.res + H.index;
        if (tid == 0) {
          long long kv = -1;
          double mv = 0.0, rv = 0.0;
          if (nb > 0) {
            const int kl = (int)(k - C_pre);
            // M_vir: (k+1) m0 in FP64 for a uniform mass, else the exact sum
            const long long mkx = unim ? 0 : mc[sw(kl, mask)];
            const double mk = unim ? double_from_fix(k + 1, 0) * L.p.m0 : double_from_fix(mkx, s_m);
            const float mkf = unim ? (float)(k + 1) * L.p.m0f : float_from_fix(mkx, s_m);
            if (k == nb - 1) status |= AHF_HALO_RVIR_BEYOND_EDGE;
            if (below_threshold(mk, mkf, rc[sw(kl, mask)], P.crit_f, P.crit)) {
              status |= AHF_HALO_RVIR_NONE;
            } else {
              kv = k;
              mv = mk;
              rv = virial_radius(mk, P.inv_crit);
              if (P.rise_edge && k == nb - 1) {
                // bound position p of the cluster: rank q holds [pre_q, pre_q + nb_loc_q)
                auto at = [&](long long p, double& r, double& m) {
                  int q = 0;
                  long long pre = 0;
                  if constexpr (CS > 1) {
                    for (; q < CS - 1; ++q) {
                      const long long nl = Cl<CS>::at(&X, q)->nb_loc;
                      if (p < pre + nl) break;
                      pre += nl;
                    }
                  }
                  const int l = sw((int)(p - pre), mask);
                  r = float_to_double(Cl<CS>::at(rc, q)[l]);
                  m = unim ? double_from_fix(p + 1, 0) * L.p.m0 : double_from_fix(Cl<CS>::at(mc, q)[l], s_m);
                };
                const long long ke = rise_edge_index(nb, at);
                if (ke >= 0) {
                  at(ke, rv, mv);
                  kv = ke;
                  status |= AHF_HALO_RISE_EDGE;
                }
              }
            }
          }
          R->n_bound = nb;
          R->n_member = n_mem;
          R->part_iter = part_iter;
          R->n_band = n_band;
          R->k_vir = kv;
          R->n_iter = n_iter;
          R->status = status;
          R->m_vir = mv;
          R->r_vir = rv;
          S.rvir = rv;
          if constexpr (CS > 1) {
            X.rvir = rv;
            X.has_rvir = 1;
          }
        } else if (tid == 32 || tid == 64 || tid == 96) {
          const int c = tid / 32 - 1;
          R->vbulk[c] = nb > 0 ? quotient(double_from_fix(S.mv[c], s_v), double_from_fix(S.c_tot[0], s_m)) : 0.0;
        }
      }
      if constexpr (CS > 1) {
        if (L.rows.prof && L.rows.n_bins <= FUSE_BINS) {
          // rows of a halo spread over the cluster: each CTA counts its chunk
          // of the radial order at every edge; rank 0 adds the counts and
          // takes the largest inclusive mass (the last particle inside)
          if (tid == 0) {
            if (!owner) X.has_rvir = 0;
            X.last_r = C_loc > 0 ? rc[sw((int)C_loc - 1, mask)] : 0.0f;
          }
          Cl<CS>::sync();
          double r_vir = 0.0;
          float r_last = 0.0f;
          for (int r2 = 0; r2 < CS; ++r2) {
            const Xchg* Y = Cl<CS>::at(&X, r2);
            if (Y->has_rvir) r_vir = Y->rvir;
            if (Y->nb_loc > 0) r_last = Y->last_r;
          }
          const double r_out = r_vir > 0.0 ? r_vir : float_to_double(r_last);
          const float r_out_f = double_to_float(r_out);
          const int n = L.rows.n_bins;
          for (int b = tid; b <= n; b += NT) {
            const float ef = b == n ? r_out_f : r_out_f * L.rows.factor_f[b];
            const double fac = b == n ? 1.0 : L.rows.factor[b];
            int lo = 0, hi = (int)C_loc;            // first local k with rc[k] > e_b
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (le_edge_band(rc[sw(mid, mask)], ef, r_out, fac)) lo = mid + 1;
              else hi = mid;
            }
            X.pc[b] = lo;
            X.pm[b] = lo > 0 ? mc[sw(lo - 1, mask)] : 0;
          }
          Cl<CS>::sync();
          if (rank == 0) {
            double* out = L.rows.prof + (size_t)H.index * n * 4;
            const float inv_r = 1.0f / r_out_f;
            for (int b = tid; b < n; b += NT) {
              long long c0 = 0, c1 = 0, f0 = 0, f1 = 0;
              for (int r2 = 0; r2 < CS; ++r2) {
                const Xchg* Y = Cl<CS>::at(&X, r2);
                c0 += Y->pc[b];
                c1 += Y->pc[b + 1];
                f0 = max(f0, Y->pm[b]);
                f1 = max(f1, Y->pm[b + 1]);
              }
              if (nb == 0) {
                out[4 * b + 0] = out[4 * b + 1] = out[4 * b + 2] = out[4 * b + 3] = 0.0;
                continue;
              }
              double M1, Ms;
              if (unim) {
                M1 = double_from_fix(c1, 0) * L.p.m0;
                Ms = double_from_fix(c1 - c0, 0) * L.p.m0;
              } else {
                M1 = double_from_fix(f1, s_m);
                Ms = double_from_fix(f1 - f0, s_m);
              }
              out[4 * b + 0] = double_from_fix(c1 - c0, 0);
              out[4 * b + 1] = M1;
              out[4 * b + 2] = shell_density(Ms, r_out, inv_r, L.rows.factor, L.rows.factor_f, n, b);
              out[4 * b + 3] = circular_velocity(P.G, P.Gf, M1, r_out, inv_r, L.rows.factor, L.rows.factor_f, n, b);
            }
          }
        }
      }
      if constexpr (CS == 1) {
        if (L.rows.prof) {
          __syncthreads();                        // S.rvir
          profile_rows(L.rows, H.index, rc, mc, [&](long long kk) { return sw((int)kk, mask); }, nb, S.rvir, s_m,
                       P.G, P.Gf, unim ? &L.p.m0 : nullptr, tid, NT);
        }
      }
    }
    if (tid == 0 && rank == 0 && L.trace) {
      long long* t = L.trace + (size_t)H.index * AHF_TRACE_FIELDS;
      t[5] = global_ns();
      t[6] = sm_id();
      t[7] = L.variant + 256ll * n_iter;
    }
    Cl<CS>::sync();
  }
}

// Dynamic shared memory: six 4-byte arrays of CAP slots, then the sort's
// counters (per-warp digit counts in a cluster, count_sort's words in one CTA).
template <int NT, int CAP, int CS>
constexpr size_t dyn_bytes() {
  return (size_t)CAP * 24 + (CS == 1 ? (size_t)count_sort_words(NT) * 4 : (size_t)(NT / 32) * 256 * 2);
}

template <int CS>
void cluster_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr) {
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

template <int NT, int CAP, int CT, int CS>
cudaError_t launch_variant(const OnchipLaunch& L, int grid, cudaStream_t s) {
  auto k = unbind_kernel<NT, CAP, CT, CS>;
  constexpr size_t smem = dyn_bytes<NT, CAP, CS>();
  static std::atomic<unsigned long long> attrs_set{0};
  if (first_use_on_device(attrs_set)) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (CS > 8) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    mark_used_on_device(attrs_set);
  }
  if constexpr (CS == 1) {
    k<<<grid, NT, smem, s>>>(L);
    return cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cluster_config<CS>(cfg, attr);
    return cudaLaunchKernelEx(&cfg, k, L);
  }
}

// CTAs of the variant that can be resident at once (whole clusters only).
template <int NT, int CAP, int CS>
int max_grid_variant(int device) {
  auto k = unbind_kernel<NT, CAP, AHF_COORD_F32_REL, CS>;
  constexpr size_t smem = dyn_bytes<NT, CAP, CS>();
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if constexpr (CS == 1) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    return per_sm * sms;
  } else {
    if (CS > 8) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(CS * (sms / CS)), 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    cluster_config<CS>(cfg, attr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess) {
      cudaGetLastError();
      clusters = 0;
    }
    return clusters * CS;
  }
}

}  // namespace

// Variants: 0 = 1 CTA x 128 threads / 1024 slots, 1 = 1 x 256 / 4096,
// 2 = 1 x 512 / 8192, 3/4/5/6 = clusters of 2/4/8/16 CTAs x 512 / 8192 slots.
int onchip_cluster_size(int variant) {
  switch (variant) {
    case 3: return 2;
    case 4: return 4;
    case 5: return 8;
    case 6: return 16;
    default: return 1;
  }
}

int onchip_capacity(int variant) {
  switch (variant) {
    case 0: return 1024;
    case 1: return 4096;
    case 2: return 8192;
    case 3: return 2 * 8192;
    case 4: return 4 * 8192;
    case 5: return 8 * 8192;
    case 6: return 16 * 8192;
    default: return 0;
  }
}

int onchip_max_grid(int variant, int device) {
  switch (variant) {
    case 0: return max_grid_variant<128, 1024, 1>(device);
    case 1: return max_grid_variant<256, 4096, 1>(device);
    case 2: return max_grid_variant<512, 8192, 1>(device);
    case 3: return max_grid_variant<512, 8192, 2>(device);
    case 4: return max_grid_variant<512, 8192, 4>(device);
    case 5: return max_grid_variant<512, 8192, 8>(device);
    case 6: return max_grid_variant<512, 8192, 16>(device);
    default: return 0;
  }
}

cudaError_t launch_onchip(const OnchipLaunch& L, int variant, int grid, cudaStream_t s) {
  const bool f64 = L.p.coord_type == AHF_COORD_F64;
  switch (variant) {
    case 0: return f64 ? launch_variant<128, 1024, AHF_COORD_F64, 1>(L, grid, s)
                       : launch_variant<128, 1024, AHF_COORD_F32_REL, 1>(L, grid, s);
    case 1: return f64 ? launch_variant<256, 4096, AHF_COORD_F64, 1>(L, grid, s)
                       : launch_variant<256, 4096, AHF_COORD_F32_REL, 1>(L, grid, s);
    case 2: return f64 ? launch_variant<512, 8192, AHF_COORD_F64, 1>(L, grid, s)
                       : launch_variant<512, 8192, AHF_COORD_F32_REL, 1>(L, grid, s);
    case 3: return f64 ? launch_variant<512, 8192, AHF_COORD_F64, 2>(L, grid, s)
                       : launch_variant<512, 8192, AHF_COORD_F32_REL, 2>(L, grid, s);
    case 4: return f64 ? launch_variant<512, 8192, AHF_COORD_F64, 4>(L, grid, s)
                       : launch_variant<512, 8192, AHF_COORD_F32_REL, 4>(L, grid, s);
    case 5: return f64 ? launch_variant<512, 8192, AHF_COORD_F64, 8>(L, grid, s)
                       : launch_variant<512, 8192, AHF_COORD_F32_REL, 8>(L, grid, s);
    case 6: return f64 ? launch_variant<512, 8192, AHF_COORD_F64, 16>(L, grid, s)
                       : launch_variant<512, 8192, AHF_COORD_F32_REL, 16>(L, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ahf
