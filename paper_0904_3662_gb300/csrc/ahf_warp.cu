// Warp class: one warp unbinds one small halo (at most WARP_CAP candidates)
// in its own slice of shared memory, with warp-level sort and scans only.
//
// The steps are those of the CTA classes (Sect. 2.1, Appendix A): gather and
// recentre, one stable radix sort by radius, the iteration of exact M(<r) and
// sum m/r prefixes -> phi -> escape test -> removal until nothing changes,
// then the bound list, phi and the virial crossing (Sect. 2.1, Eqs. 1-2).
// Small haloes are most of a halo population; giving each its own warp
// removes every CTA-wide barrier from their path, and a CTA's warps work on
// different haloes, each pulling the next one from the class's counter.
#include <cstdint>

#include "ahf_device.cuh"

namespace ahf {
namespace {

constexpr int WARP_CAP = 512;                 // candidate slots per warp
constexpr int IPL = WARP_CAP / 32;            // items per lane
constexpr int WPB = 8;                        // warps per CTA
constexpr size_t WARP_BYTES = (size_t)WARP_CAP * 24 + 256 * 2;

__device__ __forceinline__ int sw(int p, int mask) { return p ^ ((p >> 5) & mask); }

__device__ __forceinline__ long long warp_excl(long long x, int lane, long long& total) {
  const long long inc = warp_inclusive_scan(x, lane);
  total = __shfl_sync(FULL_MASK, inc, 31);
  return inc - x;
}

// Stable LSD radix sort of n <= WARP_CAP (key, val) pairs by one warp, 8-bit
// digits ranked by lane matching; the last pass writes element p at
// sw(p, mask).  For one warp this is faster than the CTA classes' counting
// sort (4 passes at most instead of 6); keys are read again for the scatter,
// so only the ranks stay in registers.  Returns 0 if the result is in
// (kA, vA), 1 if in (kB, vB).
__device__ int warp_radix_sort(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, uint16_t* hist, int n,
                               uint32_t diff, int mask, int lane) {
  int passes[4], np = 0;
  for (int d = 0; d < 4; ++d)
    if ((diff >> (8 * d)) & 0xffu) passes[np++] = d;
  if (np == 0) {
    for (int p = lane; p < n; p += 32) {
      kB[sw(p, mask)] = kA[p];
      vB[sw(p, mask)] = vA[p];
    }
    __syncwarp();
    return 1;
  }
  uint32_t *kin = kA, *vin = vA, *kout = kB, *vout = vB;
  const int nb = (n + 31) / 32;
  for (int ip = 0; ip < np; ++ip) {
    const int shift = 8 * passes[ip];
    const bool last = (ip == np - 1);
#pragma unroll
    for (int i = 0; i < 8; ++i) hist[lane * 8 + i] = 0;
    __syncwarp();
    uint16_t rk[IPL];
#pragma unroll
    for (int b = 0; b < IPL; ++b) {
      if (b < nb) {
        const int e = b * 32 + lane;
        const bool valid = e < n;
        const uint32_t key = valid ? kin[e] : 0u;
        const unsigned vmask = __ballot_sync(FULL_MASK, valid);
        rk[b] = 0;
        if (valid) {
          const uint32_t dg = (key >> shift) & 0xffu;
          const unsigned peers = __match_any_sync(vmask, dg);
          const unsigned below = peers & lanemask_lt();
          const uint16_t base = hist[dg];
          rk[b] = (uint16_t)(base + __popc(below));
          __syncwarp(vmask);
          if (below == 0) hist[dg] = (uint16_t)(base + __popc(peers));
        }
        __syncwarp();
      }
    }
    // exclusive offsets of the 256 digits (8 consecutive digits per lane)
    {
      uint32_t loc[8], s = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { loc[i] = hist[lane * 8 + i]; s += loc[i]; }
      const uint32_t inc = warp_inclusive_scan(s, lane);
      uint32_t run = inc - s;
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 8; ++i) { hist[lane * 8 + i] = (uint16_t)run; run += loc[i]; }
      __syncwarp();
    }
#pragma unroll
    for (int b = 0; b < IPL; ++b) {
      if (b < nb) {
        const int e = b * 32 + lane;
        if (e < n) {
          const uint32_t key = kin[e], val = vin[e];
          const uint32_t dg = (key >> shift) & 0xffu;
          int dst = (int)hist[dg] + (int)rk[b];
          if (last) dst = sw(dst, mask);
          kout[dst] = key;
          vout[dst] = val;
        }
      }
    }
    __syncwarp();
    uint32_t* t;
    t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
  }
  return (kin == kA) ? 0 : 1;
}

template <int CT>
__global__ void __launch_bounds__(WPB * 32) warp_kernel(OnchipLaunch L) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = dyn + (size_t)warp * WARP_BYTES;
  uint32_t* kA = (uint32_t*)base;
  uint32_t* vA = kA + WARP_CAP;
  uint32_t* kB = vA + WARP_CAP;
  uint32_t* vB = kB + WARP_CAP;
  float* ex1 = (float*)(vB + WARP_CAP);
  float* ex2 = ex1 + WARP_CAP;
  uint16_t* hist = (uint16_t*)(ex2 + WARP_CAP);
  const ParamsDev& P = L.prm;

  for (;;) {
    int hq = 0;
    if (lane == 0) hq = atomicAdd(L.queue, 1);
    hq = __shfl_sync(FULL_MASK, hq, 0);
    if (hq >= L.n_halos) break;
    const HaloDev H = L.halos[hq];
    if (lane == 0) trace_mark(L.trace, H.index, 0);
    const int n_cand = (int)H.count;
    if (n_cand > WARP_CAP) {       // the scheduler never does this; report, do not overrun
      if (lane == 0) atomicOr(L.out.err, ERR_CAPACITY);
      continue;
    }
    prefetch_candidates<CT>(L.p, L.out.member_idx, H.offset, H.offset + n_cand, lane);
    int ipt = 1;
    while (ipt * 32 < n_cand) ipt <<= 1;
    const int mask = ipt - 1;

    // ---- gather ----
    uint32_t orb = 0u, andb = 0xffffffffu, mxm = 0u, mxr = 0u, mxv = 0u;
    int nmem = 0;
    for (int i = lane; i < n_cand; i += 32) {
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
        float df[3];
        offset_of<CT>(L.p, pi, H, df, f);
        if (member_of<CT>(L.p, pi, H, df, f)) {
          const float r = radius_of(df);
          key = __float_as_uint(r);
          const float m = load_mass<CT>(L.p, pi);
          float v[3];
          load_velocity<CT>(L.p, pi, v);
          if (L.rec) put_record(L.rec + 2 * (H.gbase + i), df, m, v);
          mxm = max(mxm, __float_as_uint(fabsf(m)));
          mxr = max(mxr, __float_as_uint(fabsf(m * rinv_of(r, P.r_soft_f))));
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
    const int n_mem = (int)__reduce_add_sync(FULL_MASK, (unsigned)nmem);
    __syncwarp();
    const int s_m = fix_scale(float_exponent_of_bits(mxm), n_mem);
    const int s_r = fix_scale(float_exponent_of_bits(mxr), n_mem);
    const int s_v = fix_scale(float_exponent_of_bits(mxv), n_mem);
    const bool unim = L.p.m == nullptr;                  // every particle has mass m0
    const long long m0fix = fix_from_float(L.p.m0f, s_m);
    // 2^-s of the mass and m/r sums as floats (0 when not normal): each
    // exact sum's float value is then one multiply, the bits of float_from_fix
    const float sc_m = pow2_neg(s_m), sc_r = pow2_neg(s_r);

    if (lane == 0) trace_mark(L.trace, H.index, 1);
    // ---- radial sort (once) ----
    const int which = warp_radix_sort(kA, vA, kB, vB, hist, n_cand, orb ^ andb, mask, lane);
    float* rr = (float*)(which ? kB : kA);
    uint32_t* jj = which ? vB : vA;
    float* mm = (float*)(which ? kA : kB);
    float* wx = (float*)(which ? vA : vB);
    float* wy = ex1;
    float* wz = ex2;

    if (lane == 0) trace_mark(L.trace, H.index, 2);
    // ---- fill ----
    long long mv[3] = {0, 0, 0};
    for (int p = lane; p < n_mem; p += 32) {
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
      for (int k = 0; k < 3; ++k) mv[k] += fix_from_float(__fmul_rn(m, v[k]), s_v);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) mv[k] = warp_sum(mv[k]);
    __syncwarp();

    const int p0 = lane * ipt;
    long long tm_own = 0, tr_own = 0, tc_own = 0;
    for (int k = 0; k < ipt; ++k) {
      const int p = p0 + k;
      if (p < n_mem) {
        const int q = sw(p, mask);
        const float mq = mm[q];
        const float m = unim ? L.p.m0f : mq;
        const float ri = unim ? mq : rinv_of(rr[q], P.r_soft_f);
        tm_own += (unim ? m0fix : fix_from_float(m, s_m));
        tr_own += fix_from_float(m * ri, s_r);
        tc_own += 1;
      }
    }

    if (lane == 0) trace_mark(L.trace, H.index, 3);
    // ---- iterate (Appendix A) ----
    int n_iter = 0, status = 0;
    long long part_iter = 0, n_band = 0;
    int n_alive = n_mem;
    bool converged = false;
    float vb0 = 0.0f, vb1 = 0.0f, vb2 = 0.0f;
    while (n_alive > 0 && n_iter < P.max_iter) {
      ++n_iter;
      part_iter += n_alive;
      long long M_tot, T_tot;
      long long tm = warp_excl(tm_own, lane, M_tot);
      long long tr = warp_excl(tr_own, lane, T_tot);
      // v_bulk of the current set (of the initial set with AHF_VAR_VBULK_INITIAL)
      if (n_iter == 1 || !P.vbulk_initial) {
        const float mt = float_from_fix(M_tot, s_m);
        vb0 = float_from_fix(mv[0], s_v) / mt;
        vb1 = float_from_fix(mv[1], s_v) / mt;
        vb2 = float_from_fix(mv[2], s_v) / mt;
      }
      long long rm = 0, rq = 0, rv0 = 0, rv1 = 0, rv2 = 0;
      int nrem = 0, nband = 0;
      uint32_t rmask = 0;                 // this lane's removals (bit k: position p0 + k)
      // no branch per member: a slot past the members or removed earlier
      // adds nothing and is not tested (every slot of the run is within the
      // arrays), so the loop's members can overlap
      if (p0 < n_mem) {
#pragma unroll 4
        for (int k = 0; k < ipt; ++k) {
          const int p = p0 + k;
          const int q = sw(p, mask);
          const float mq = mm[q];
          const bool alive = p < n_mem && !signbit(mq);
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
      // the removed, off the per-particle path: exact m v from the stored
      // velocity, and their removal iteration
      for (uint32_t b = rmask; b; b &= b - 1) {
        const int k = __ffs(b) - 1;
        const int q = sw(p0 + k, mask);
        const float m = unim ? L.p.m0f : -mm[q];
        const long long slot = H.offset + (long long)jj[q];
        float v[3];
        if (L.rec) get_velocity_record(L.rec + 2 * (H.gbase + (long long)jj[q]), v);
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
      const int removed = (int)__reduce_add_sync(FULL_MASK, (unsigned)nrem);
      n_band += (int)__reduce_add_sync(FULL_MASK, (unsigned)nband);
      if (removed) {
        mv[0] -= warp_sum(rv0);
        mv[1] -= warp_sum(rv1);
        mv[2] -= warp_sum(rv2);
      }
      n_alive -= removed;
      if (removed == 0) { converged = true; break; }
    }
    if (n_alive == 0) status |= AHF_HALO_EMPTY;
    else if (!converged) status |= AHF_HALO_NOT_CONVERGED;

    if (lane == 0) trace_mark(L.trace, H.index, 4);
    // ---- emit ----
    float* rc = wx;
    long long* mc = (long long*)ex1;      // ex1 and ex2 are contiguous
    long long M_tot, T_tot, nb;
    long long tm = warp_excl(tm_own, lane, M_tot);
    long long tr = warp_excl(tr_own, lane, T_tot);
    long long tl = warp_excl(tc_own, lane, nb);
    __syncwarp();
    for (int k = 0; k < ipt; ++k) {
      const int p = p0 + k;
      if (p < n_mem) {
        const int q = sw(p, mask);
        const float mq = mm[q];
        if (!signbit(mq)) {
          const float r = rr[q];
          const float m = unim ? L.p.m0f : mq;
          const float ri = unim ? mq : rinv_of(r, P.r_soft_f);
          const long long mfix = (unim ? m0fix : fix_from_float(m, s_m));
          const float phi = phi_of(fix_to_float_fast(tm, s_m, sc_m), ri, fix_to_float_fast(T_tot - tr, s_r, sc_r),
                                   P.Gf);
          const long long slot = H.offset + (long long)jj[q];
          const long long pi = L.out.member_idx ? L.out.member_idx[slot] : slot;
          const long long dst = H.offset + tl;
          L.out.bound_idx[dst] = pi;
          if (L.out.phi) ((float*)L.out.phi)[dst] = phi;
          if (L.out.removed_iter) L.out.removed_iter[slot] = 0;
          const int kq = sw((int)tl, mask);
          rc[kq] = r;
          mc[kq] = tm + mfix;
          tm += mfix;
          tr += fix_from_float(m * ri, s_r);
          tl += 1;
        }
      }
    }
    __syncwarp();
    // virial: first k with M_k < delta_rho 4pi/3 r_{k+1}^3 (r_{N+1} = inf)
    int kf = 0x7fffffff;
    for (int k = 0; k < ipt; ++k) {
      const int kk = p0 + k;
      if (kk < nb) {
        bool cross = true;
        if (kk + 1 < nb) {
          const float rn = rc[sw(kk + 1, mask)];
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
        if (cross) { kf = kk; break; }
      }
    }
    kf = (int)__reduce_min_sync(FULL_MASK, (unsigned)kf);
    // the record: lane 0 the virial pair, lanes 1-3 one bulk velocity
    // component each (FP64 work in parallel rather than in sequence)
    double r_vir_l = 0.0;
    if (lane == 0) {
      long long kv = -1;
      double mvir = 0.0;
      if (nb > 0) {
        // M_vir: (k+1) m0 in FP64 for a uniform mass, else the exact sum
        const long long mkx = unim ? 0 : mc[sw(kf, mask)];
        const double mk = unim ? double_from_fix(kf + 1, 0) * L.p.m0 : double_from_fix(mkx, s_m);
        const float mkf = unim ? (float)(kf + 1) * L.p.m0f : float_from_fix(mkx, s_m);
        if (kf == nb - 1) status |= AHF_HALO_RVIR_BEYOND_EDGE;
        if (below_threshold(mk, mkf, rc[sw(kf, mask)], P.crit_f, P.crit)) {
          status |= AHF_HALO_RVIR_NONE;
        } else {
          kv = kf;
          mvir = mk;
          r_vir_l = virial_radius(mk, P.inv_crit);
          if (P.rise_edge && kf == nb - 1) {
            auto at = [&](long long k, double& r, double& m) {
              r = float_to_double(rc[sw((int)k, mask)]);
              m = unim ? double_from_fix(k + 1, 0) * L.p.m0 : double_from_fix(mc[sw((int)k, mask)], s_m);
            };
            const long long ke = rise_edge_index(nb, at);
            if (ke >= 0) {
              at(ke, r_vir_l, mvir);
              kv = ke;
              status |= AHF_HALO_RISE_EDGE;
            }
          }
        }
      }
      ahf_result* R = L.out.res + H.index;
      R->n_bound = nb;
      R->n_member = n_mem;
      R->part_iter = part_iter;
      R->n_band = n_band;
      R->k_vir = kv;
      R->n_iter = n_iter;
      R->status = status;
      R->m_vir = mvir;
      R->r_vir = r_vir_l;
    } else if (lane < 4) {
      const long long m = lane == 1 ? mv[0] : (lane == 2 ? mv[1] : mv[2]);
      L.out.res[H.index].vbulk[lane - 1] = nb > 0 ? quotient(double_from_fix(m, s_v), double_from_fix(M_tot, s_m)) : 0.0;
    }
    if (L.rows.prof) {
      const double r_vir = __shfl_sync(FULL_MASK, r_vir_l, 0);
      profile_rows(L.rows, H.index, rc, mc, [&](long long k) { return sw((int)k, mask); }, nb, r_vir, s_m, P.G, P.Gf,
                   unim ? &L.p.m0 : nullptr, lane, 32);
    }
    if (lane == 0 && L.trace) {
      long long* t = L.trace + (size_t)H.index * AHF_TRACE_FIELDS;
      t[5] = global_ns();
      t[6] = sm_id();
      t[7] = L.variant + 256ll * n_iter;
    }
    __syncwarp();
  }
}

template <int CT>
cudaError_t launch_ct(const OnchipLaunch& L, int grid, cudaStream_t s) {
  auto k = warp_kernel<CT>;
  constexpr size_t smem = WARP_BYTES * WPB;
  static std::atomic<unsigned long long> attrs_set{0};
  if (first_use_on_device(attrs_set)) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mark_used_on_device(attrs_set);
  }
  k<<<grid, WPB * 32, smem, s>>>(L);
  return cudaGetLastError();
}

}  // namespace

int warp_capacity() { return WARP_CAP; }

// Resident warps (= haloes in flight) of the warp class; the launch grid is
// in CTAs of WPB warps.
int warp_max_grid(int device) {
  auto k = warp_kernel<AHF_COORD_F32_REL>;
  constexpr size_t smem = WARP_BYTES * WPB;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, WPB * 32, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}

int warp_halos_per_cta() { return WPB; }

cudaError_t launch_warp(const OnchipLaunch& L, int grid, cudaStream_t s) {
  return L.p.coord_type == AHF_COORD_F64 ? launch_ct<AHF_COORD_F64>(L, grid, s)
                                         : launch_ct<AHF_COORD_F32_REL>(L, grid, s);
}

}  // namespace ahf
