// Log-radial profiles of bound sets (Sect. 2.1: the radially binned halo
// output built from the bound particle lists).
//
// Bin b of a halo covers (e_b, e_{b+1}], e_b = r_out f^(1 - b/n), r_out the
// virial radius (or the outermost bound radius when there is none).  The
// factors f^(1 - b/n) are computed once per call on the host; a halo's edges
// are r_out times them.  The bound list is cut into fixed chunks; each CTA
// bins one chunk (radius recomputed from the particle store exactly as the
// unbinding kernels do).  The bin of a float radius is decided against the
// FP64 edge: comparisons against the edge rounded to float are exact except
// when the radius equals that rounded edge, which is then settled in FP64.
// A halo held by one chunk gets its rows from that CTA; otherwise a second
// kernel adds the chunk partials in chunk order.  Columns:
//   count, M(<= e_{b+1}), shell density, sqrt(G M(<= e_{b+1}) / e_{b+1}).
// With a uniform particle mass the masses are count * m0 exactly.
#include <cstdint>

#include "ahf_device.cuh"

namespace ahf {
namespace {

constexpr int PT = 256;
constexpr int MAX_BINS = 4096;

template <int CT>
__device__ __forceinline__ float bound_radius(const ProfileLaunch& L, const HaloDev& H, long long pi) {
  long long f[3];
  float df[3];
  offset_of<CT>(L.p, pi, H, df, f);
  return radius_of(df);
}

// Inclusive block scan of one double per thread (PT threads).
__device__ __forceinline__ double block_scan_incl(double x, double* wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  double b = 0.0;
  for (int w = 0; w < warp; ++w) b += wsum[w];
  __syncthreads();
  return x + b;
}

// Rows of one halo from its per-bin counts and masses (held in shared
// memory), written by the whole CTA.
__device__ void write_rows(const ProfileLaunch& L, int h, const double* e, const unsigned long long* cnt,
                           const double* mass, double inner) {
  __shared__ double wsum[PT / 32];
  __shared__ double carry;
  const int n = L.n_bins;
  double* out = L.prof + (size_t)h * n * 4;
  const double r_out = e[n];
  const float inv_r = 1.0f / double_to_float(r_out);
  if (threadIdx.x == 0) carry = inner;
  __syncthreads();
  for (int b0 = 0; b0 < n; b0 += PT) {
    const int b = b0 + threadIdx.x;
    const double mb = b < n ? mass[b] : 0.0;
    const double inc = block_scan_incl(mb, wsum);
    const double run = carry + inc;
    if (b < n) {
      out[4 * b + 0] = (double)cnt[b];
      out[4 * b + 1] = run;
      out[4 * b + 2] = shell_density(mb, r_out, inv_r, L.edge_factor, L.edge_factor_f, n, b);
      out[4 * b + 3] = circular_velocity(L.prm.G, L.prm.Gf, run, r_out, inv_r, L.edge_factor, L.edge_factor_f, n, b);
    }
    __syncthreads();
    if (threadIdx.x == PT - 1) carry = run;
    __syncthreads();
  }
}

// chunk_acc layout per chunk: [0] inner mass (bits of double), [1] inner
// count, [2 + 2b] count, [3 + 2b] mass (bits of double)
template <int CT>
__global__ void __launch_bounds__(PT) prof_chunk(ProfileLaunch L, const int* __restrict__ halo_chunk0) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int n = L.n_bins;
  double* e = (double*)dsm;                                        // n + 1 edges
  double* mb = e + (n + 1);                                        // n masses
  unsigned long long* cb = (unsigned long long*)(mb + n);          // n counts
  float* ef = (float*)(cb + n);                                    // n + 1 float edges
  __shared__ double inner;
  __shared__ unsigned long long cinner;
  __shared__ float r_last;
  const int c = blockIdx.x;
  const int h = L.chunk_halo[c];
  const HaloDev H = L.halos[h];
  const long long start = L.chunk_start[c];
  const long long nb = L.res[h].n_bound;
  const double rvir = L.res[h].r_vir;
  const bool single = halo_chunk0[h + 1] - halo_chunk0[h] == 1;
  long long* acc = L.chunk_acc + (size_t)c * (2 + 2 * n);
  if (start >= nb && !single) {
    for (int i = threadIdx.x; i < 2 + 2 * n; i += PT) acc[i] = 0;
    return;
  }
  if (nb == 0) {                                                   // empty halo, single chunk
    double* out = L.prof + (size_t)h * n * 4;
    for (int i = threadIdx.x; i < 4 * n; i += PT) out[i] = 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    inner = 0.0;
    cinner = 0ull;
    r_last = rvir > 0.0 ? 0.0f : bound_radius<CT>(L, H, L.bound_idx[H.offset + nb - 1]);
  }
  for (int b = threadIdx.x; b < n; b += PT) { mb[b] = 0.0; cb[b] = 0ull; }
  __syncthreads();
  const double r_out = rvir > 0.0 ? rvir : (double)r_last;
  for (int b = threadIdx.x; b <= n; b += PT) {
    e[b] = b == n ? r_out : r_out * L.edge_factor[b];
    ef[b] = (float)e[b];
  }
  __syncthreads();
  const float rof = (float)r_out;
  const float inv_lnf = 1.0f / logf((float)L.r_min_frac);
  const long long end = min(nb, start + (long long)PROFILE_CHUNK);
  double my_inner = 0.0;
  unsigned long long my_ci = 0;
  for (long long k = start + threadIdx.x; k < end; k += PT) {
    const long long pi = L.bound_idx[H.offset + k];
    const float r = bound_radius<CT>(L, H, pi);
    if (!le_edge(r, ef[n], e[n])) continue;                        // beyond r_out
    double m = L.p.m0;
    if (L.p.m) m = CT == AHF_COORD_F64 ? __ldg((const double*)L.p.m + pi) : (double)__ldg((const float*)L.p.m + pi);
    if (le_edge(r, ef[0], e[0])) {                                 // inside the innermost edge
      ++my_ci;
      if (L.p.m) my_inner += m;
      continue;
    }
    // guess from the logarithm, then settle against the edges
    int b = (int)floorf((float)n * (1.0f - __logf(r / rof) * inv_lnf));
    b = max(0, min(n - 1, b));
    while (b > 0 && le_edge(r, ef[b], e[b])) --b;
    while (b < n - 1 && !le_edge(r, ef[b + 1], e[b + 1])) ++b;
    atomicAdd(&cb[b], 1ull);
    if (L.p.m) atomicAdd(&mb[b], m);
  }
  for (int o = 16; o > 0; o >>= 1) my_ci += __shfl_xor_sync(FULL_MASK, my_ci, o);
  if ((threadIdx.x & 31) == 0 && my_ci) atomicAdd(&cinner, my_ci);
  if (L.p.m && my_inner != 0.0) atomicAdd(&inner, my_inner);
  __syncthreads();
  if (!L.p.m) {
    if (threadIdx.x == 0) inner = (double)cinner * L.p.m0;
    for (int b = threadIdx.x; b < n; b += PT) mb[b] = (double)cb[b] * L.p.m0;
  }
  __syncthreads();
  if (single) {
    write_rows(L, h, e, cb, mb, inner);
    return;
  }
  if (threadIdx.x == 0) {
    acc[0] = __double_as_longlong(inner);
    acc[1] = (long long)cinner;
  }
  for (int b = threadIdx.x; b < n; b += PT) {
    acc[2 + 2 * b] = (long long)cb[b];
    acc[3 + 2 * b] = __double_as_longlong(mb[b]);
  }
}

// One CTA per halo held by several chunks: add the partials in chunk order.
template <int CT>
__global__ void __launch_bounds__(PT) prof_final(ProfileLaunch L, const int* __restrict__ halo_chunk0) {
  const int h = blockIdx.x;
  const int c0 = halo_chunk0[h], c1 = halo_chunk0[h + 1];
  if (c1 - c0 <= 1) return;                                        // done by the chunk kernel
  const int n = L.n_bins;
  extern __shared__ __align__(16) unsigned char dsm[];
  double* e = (double*)dsm;
  double* mass = e + (n + 1);
  unsigned long long* cnt = (unsigned long long*)(mass + n);
  __shared__ double inner;
  __shared__ float r_last;
  const long long nb = L.res[h].n_bound;
  const double rvir = L.res[h].r_vir;
  if (nb == 0) {
    double* out = L.prof + (size_t)h * n * 4;
    for (int i = threadIdx.x; i < 4 * n; i += PT) out[i] = 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    const HaloDev H = L.halos[h];
    r_last = rvir > 0.0 ? 0.0f : bound_radius<CT>(L, H, L.bound_idx[H.offset + nb - 1]);
    double in = 0.0;
    for (int c = c0; c < c1; ++c) in += __longlong_as_double(L.chunk_acc[(size_t)c * (2 + 2 * n)]);
    inner = in;
  }
  __syncthreads();
  const double r_out = rvir > 0.0 ? rvir : (double)r_last;
  for (int b = threadIdx.x; b <= n; b += PT) e[b] = b == n ? r_out : r_out * L.edge_factor[b];
  for (int b = threadIdx.x; b < n; b += PT) {
    unsigned long long cc = 0;
    double mm = 0.0;
    for (int c = c0; c < c1; ++c) {
      const long long* acc = L.chunk_acc + (size_t)c * (2 + 2 * n);
      cc += (unsigned long long)acc[2 + 2 * b];
      mm += __longlong_as_double(acc[3 + 2 * b]);
    }
    cnt[b] = cc;
    mass[b] = mm;
  }
  __syncthreads();
  write_rows(L, h, e, cnt, mass, inner);
}

}  // namespace

int profile_max_bins() { return MAX_BINS; }

cudaError_t launch_profile(const ProfileLaunch& L, const int* halo_chunk0, cudaStream_t s) {
  const size_t sm1 = (size_t)(L.n_bins + 1) * 8 + (size_t)L.n_bins * 16 + (size_t)(L.n_bins + 1) * 4 + 16;
  const size_t sm2 = (size_t)(L.n_bins + 1) * 8 + (size_t)L.n_bins * 16;
  const bool f64 = L.p.coord_type == AHF_COORD_F64;
  cudaError_t e;
  if (L.n_chunks > 0) {
    auto k = f64 ? prof_chunk<AHF_COORD_F64> : prof_chunk<AHF_COORD_F32_REL>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    k<<<L.n_chunks, PT, sm1, s>>>(L, halo_chunk0);
  }
  if (L.n_multi > 0) {
    auto k = f64 ? prof_final<AHF_COORD_F64> : prof_final<AHF_COORD_F32_REL>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    if (e != cudaSuccess) return e;
    k<<<L.n_halos, PT, sm2, s>>>(L, halo_chunk0);
  }
  return cudaGetLastError();
}

}  // namespace ahf
