// Integral properties of bound sets (Sect. 3.1: the spin parameter
// lambda = J sqrt|E| / (G M^(5/2)); the rotation curve's peak) and the
// cross-identification of two catalogues by xi = N_shared^2 / (N_1 N_2)
// (Sect. 3.2).
//
// Properties.  A halo's material within r_vir is its bound list up to k_vir
// (the whole list without an r_vir), in radial order.  The bound lists are
// cut into fixed chunks.  Pass 1 (one CTA per chunk) accumulates the moments
//   S_m, S_mv, S_md, S_m(d x v), S_m|w|^2, S_mw (w = v + H d), S_m phi
// in FP64; with v_bar = S_mv / M they give J = S_m(d x v) - S_md x v_bar and
// K = (S_m|w|^2 - 2 v_bar . S_mw + M |v_bar|^2) / 2 = sum m |w - v_bar|^2 / 2.
// Pass 2 (per chunk) forms the inclusive mass M(<= r_i) from the chunk's
// offset (the earlier chunks' masses) and a block scan, and keeps the
// largest M(<= r_i) / r_i, compared as M^2 r'^2 > M'^2 r^2 (no square root per
// particle).  A final kernel adds each halo's chunks in chunk order.
//
// Matching.  Every id of the second catalogue is labelled with its halo; one
// CTA per halo of the first catalogue counts the labels of its ids in a
// shared-memory hash table and keeps the largest xi.
#include <cstdint>

#include "ahf_device.cuh"

namespace ahf {
namespace {

constexpr int PT = 256;
constexpr int PER_T = PROPS_CHUNK / PT;   // consecutive elements per thread in pass 2

__device__ __forceinline__ double block_sum_d(double x, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = warp_sum(x);
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < PT / 32; ++w) t += red[w];     // fixed order
  return t;                                            // valid in thread 0
}

// Offset from the centre in FP64 (minimum image in a periodic box), velocity
// and mass of particle pi.
template <int CT>
__device__ __forceinline__ void load_f64(const PropsLaunch& L, const HaloDev& H, long long pi, double d[3], double v[3],
                                         double& m) {
  Cand<CT> c;
  load_cand<CT>(L.p, pi, c);
  const double x[3] = {(double)c.x, (double)c.y, (double)c.z};
  const double box = L.frame.box;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double t = x[a] - H.c[a];
    if (box > 0.0) {
      const double half = 0.5 * box;
      if (t > half) t -= box;
      else if (t < -half) t += box;
    }
    d[a] = t;
  }
  v[0] = (double)c.vx;
  v[1] = (double)c.vy;
  v[2] = (double)c.vz;
  m = L.p.m ? (double)c.m : L.p.m0;
}

__device__ __forceinline__ long long n_used(const ahf_result& r) {
  return r.k_vir >= 0 ? r.k_vir + 1 : r.n_bound;
}

// Pass 1: the moments of one chunk.
template <int CT>
__global__ void __launch_bounds__(PT) props_moments(PropsLaunch L) {
  __shared__ double red[PT / 32];
  const int c = blockIdx.x;
  const int h = L.chunk_halo[c];
  const HaloDev& H = L.halos[h];
  const long long n = n_used(L.res[h]);
  const long long start = L.chunk_start[c];
  const long long end = min(n, start + (long long)PROPS_CHUNK);
  double s[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) s[k] = 0.0;
  for (long long k = start + threadIdx.x; k < end; k += PT) {
    const long long pi = L.bound_idx[H.offset + k];
    double d[3], v[3], m;
    load_f64<CT>(L, H, pi, d, v, m);
    const double phi = L.phi_f64 ? ((const double*)L.phi)[H.offset + k] : (double)((const float*)L.phi)[H.offset + k];
    double w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) w[a] = v[a] + L.H * d[a];
    s[0] += m;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s[1 + a] += m * v[a];
      s[4 + a] += m * d[a];
      s[11 + a] += m * w[a];
    }
    s[7] += m * (d[1] * v[2] - d[2] * v[1]);
    s[8] += m * (d[2] * v[0] - d[0] * v[2]);
    s[9] += m * (d[0] * v[1] - d[1] * v[0]);
    s[10] += m * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    s[14] += m * phi;
  }
  double* out = L.part + (size_t)c * PROPS_PART;
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    const double t = block_sum_d(s[k], red);
    if (threadIdx.x == 0) out[k] = t;
  }
  if (threadIdx.x == 0) out[15] = (double)max(0ll, end - start);
}

// Pass 2: the rotation-curve maximum within one chunk.
template <int CT>
__global__ void __launch_bounds__(PT) props_vmax(PropsLaunch L) {
  __shared__ double red[PT / 32];
  __shared__ double wtot[PT / 32];
  __shared__ double m_off;
  __shared__ double bm[PT], br2[PT];
  __shared__ long long bk[PT];
  const int c = blockIdx.x;
  const int h = L.chunk_halo[c];
  const HaloDev& H = L.halos[h];
  const long long n = n_used(L.res[h]);
  const long long start = L.chunk_start[c];
  const long long end = min(n, start + (long long)PROPS_CHUNK);
  // the mass of the halo's earlier chunks, added in chunk order
  double pre = 0.0;
  for (int k = L.halo_chunk0[h] + (int)threadIdx.x; k < c; k += PT) pre += L.part[(size_t)k * PROPS_PART];
  const double off = block_sum_d(pre, red);
  if (threadIdx.x == 0) m_off = off;
  // this thread's run of consecutive elements: masses and squared radii
  const long long k0 = start + (long long)threadIdx.x * PER_T;
  double m[PER_T], r2[PER_T];
  double run = 0.0;
#pragma unroll
  for (int j = 0; j < PER_T; ++j) {
    m[j] = 0.0;
    r2[j] = 0.0;
    const long long k = k0 + j;
    if (k < end) {
      double d[3], v[3];
      load_f64<CT>(L, H, L.bound_idx[H.offset + k], d, v, m[j]);
      r2[j] = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    }
    run += m[j];
  }
  // exclusive block scan of the runs' masses
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(FULL_MASK, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) wtot[warp] = inc;
  __syncthreads();
  double base = m_off;
  for (int w = 0; w < warp; ++w) base += wtot[w];
  base += inc - run;
  // the largest M(<= r_i) / r_i of the run (first one on ties)
  double best_m = 0.0, best_r2 = 0.0;
  long long best_k = -1;
  double cum = base;
#pragma unroll
  for (int j = 0; j < PER_T; ++j) {
    const long long k = k0 + j;
    cum += m[j];
    if (k < end && r2[j] > 0.0) {
      if (best_k < 0 || cum * cum * best_r2 > best_m * best_m * r2[j]) {
        best_m = cum;
        best_r2 = r2[j];
        best_k = k;
      }
    }
  }
  bm[threadIdx.x] = best_m;
  br2[threadIdx.x] = best_r2;
  bk[threadIdx.x] = best_k;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long kb = -1;
    double mb = 0.0, rb = 0.0;
    for (int t = 0; t < PT; ++t) {           // in element order: ties keep the first
      if (bk[t] < 0) continue;
      if (kb < 0 || bm[t] * bm[t] * rb > mb * mb * br2[t]) {
        kb = bk[t];
        mb = bm[t];
        rb = br2[t];
      }
    }
    double* out = L.part + (size_t)c * PROPS_PART;
    out[16] = mb;
    out[17] = rb;
    out[18] = (double)kb;
  }
}

// One thread per halo: add the chunks in order and form the properties.
__global__ void props_final(PropsLaunch L) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= L.n_halos) return;
  const ahf_result r = L.res[h];
  const long long n = n_used(r);
  double* o = L.props + (size_t)h * AHF_PROP_FIELDS;
  for (int k = 0; k < AHF_PROP_FIELDS; ++k) o[k] = 0.0;
  o[11] = r.k_vir >= 0 ? 1.0 : 0.0;
  if (n <= 0) return;
  double s[15];
  for (int k = 0; k < 15; ++k) s[k] = 0.0;
  double mb = 0.0, rb = 0.0, kb = -1.0;
  for (int c = L.halo_chunk0[h]; c < L.halo_chunk0[h + 1]; ++c) {
    const double* p = L.part + (size_t)c * PROPS_PART;
    if (p[15] <= 0.0) continue;
    for (int k = 0; k < 15; ++k) s[k] += p[k];
    if (p[18] >= 0.0 && (kb < 0.0 || p[16] * p[16] * rb > mb * mb * p[17])) {
      mb = p[16];
      rb = p[17];
      kb = p[18];
    }
  }
  const double M = s[0];
  const double vb[3] = {s[1] / M, s[2] / M, s[3] / M};
  const double J[3] = {s[7] - (s[5] * vb[2] - s[6] * vb[1]), s[8] - (s[6] * vb[0] - s[4] * vb[2]),
                       s[9] - (s[4] * vb[1] - s[5] * vb[0])};
  const double K = 0.5 * (s[10] - 2.0 * (vb[0] * s[11] + vb[1] * s[12] + vb[2] * s[13]) +
                          M * (vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]));
  const double U = 0.5 * s[14];
  const double E = K + U;
  const double Jn = sqrt(J[0] * J[0] + J[1] * J[1] + J[2] * J[2]);
  o[0] = (double)n;
  o[1] = M;
  o[2] = J[0];
  o[3] = J[1];
  o[4] = J[2];
  o[5] = K;
  o[6] = U;
  o[7] = E;
  o[8] = Jn * sqrt(fabs(E)) / (L.G * M * M * sqrt(M));
  if (kb >= 0.0) {
    const double rmax = sqrt(rb);
    o[9] = sqrt(L.G * mb / rmax);
    o[10] = rmax;
  }
}

// ---- matching ----------------------------------------------------------------

__global__ void __launch_bounds__(PT) match_label(MatchLaunch L) {
  const int b = blockIdx.x;
  const long long off = L.off_b[b], cnt = L.cnt_b[b];
  for (long long k = threadIdx.x; k < cnt; k += PT) {
    const long long id = L.ids_b[off + k];
    if (id < 0 || id >= L.n_ids) {
      atomicOr(L.err, ERR_ID_RANGE);
      continue;
    }
    const int old = atomicCAS(&L.label[id], -1, b);
    if (old != -1 && old != b) atomicOr(L.err, ERR_SHARED_ID);
  }
}

__global__ void __launch_bounds__(PT) match_best(MatchLaunch L) {
  __shared__ int key[MATCH_TABLE];
  __shared__ int cnt[MATCH_TABLE];
  __shared__ int overflow;
  __shared__ double bx[PT];
  __shared__ int bb[PT];
  const int a = blockIdx.x;
  for (int i = threadIdx.x; i < MATCH_TABLE; i += PT) {
    key[i] = -1;
    cnt[i] = 0;
  }
  if (threadIdx.x == 0) overflow = 0;
  __syncthreads();
  const long long off = L.off_a[a], na = L.cnt_a[a];
  for (long long k = threadIdx.x; k < na; k += PT) {
    const long long id = L.ids_a[off + k];
    if (id < 0 || id >= L.n_ids) {
      atomicOr(L.err, ERR_ID_RANGE);
      continue;
    }
    const int b = L.label[id];
    if (b < 0) continue;
    unsigned slot = ((unsigned)b * 2654435761u) & (MATCH_TABLE - 1);
    bool placed = false;
    for (int probe = 0; probe < MATCH_TABLE; ++probe) {   // bounded: at most every slot once
      const int k0 = atomicCAS(&key[slot], -1, b);
      if (k0 == -1 || k0 == b) {
        atomicAdd(&cnt[slot], 1);
        placed = true;
        break;
      }
      slot = (slot + 1) & (MATCH_TABLE - 1);
    }
    if (!placed) overflow = 1;
  }
  __syncthreads();
  double best_x = 0.0;
  int best_b = -1;
  for (int i = threadIdx.x; i < MATCH_TABLE; i += PT) {
    const int b = key[i];
    if (b < 0) continue;
    const double c = (double)cnt[i];
    const double x = c * c / ((double)na * (double)L.cnt_b[b]);
    if (x > best_x || (x == best_x && best_b >= 0 && b < best_b)) {
      best_x = x;
      best_b = b;
    }
  }
  bx[threadIdx.x] = best_x;
  bb[threadIdx.x] = best_b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    int b = -1;
    for (int t = 0; t < PT; ++t) {
      if (bb[t] < 0) continue;
      if (b < 0 || bx[t] > x || (bx[t] == x && bb[t] < b)) {
        x = bx[t];
        b = bb[t];
      }
    }
    long long sh = 0;
    if (b >= 0)
      for (int i = 0; i < MATCH_TABLE; ++i)
        if (key[i] == b) sh = cnt[i];
    if (overflow) {
      atomicOr(L.err, ERR_MATCH_TABLE);
      b = -2;
      x = 0.0;
      sh = 0;
    }
    L.best[a] = b;
    L.shared[a] = sh;
    L.xi[a] = b >= 0 ? x : 0.0;
  }
}

}  // namespace

cudaError_t launch_properties(const PropsLaunch& L, cudaStream_t s) {
  if (L.n_halos == 0) return cudaSuccess;
  const bool f64 = L.p.coord_type == AHF_COORD_F64;
  if (L.n_chunks > 0) {
    if (f64) {
      props_moments<AHF_COORD_F64><<<L.n_chunks, PT, 0, s>>>(L);
      props_vmax<AHF_COORD_F64><<<L.n_chunks, PT, 0, s>>>(L);
    } else {
      props_moments<AHF_COORD_F32_REL><<<L.n_chunks, PT, 0, s>>>(L);
      props_vmax<AHF_COORD_F32_REL><<<L.n_chunks, PT, 0, s>>>(L);
    }
  }
  props_final<<<(L.n_halos + 127) / 128, 128, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_match(const MatchLaunch& L, cudaStream_t s) {
  if (L.n_b > 0) match_label<<<L.n_b, PT, 0, s>>>(L);
  if (L.n_a > 0) match_best<<<L.n_a, PT, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace ahf
