// Log-radial profiles of bound sets (Sect. 2.1: the radially binned halo
// output built from the bound particle lists).
//
// Bin b of a halo covers (e_b, e_{b+1}], e_b = r_out f^(1 - b/n), r_out the
// virial radius (or the outermost bound radius when there is none).  The
// bound list is cut into fixed chunks; each CTA bins one chunk (radius
// recomputed from the particle store exactly as the unbinding kernels do,
// bin decided against FP64 edges), and a second kernel adds the chunk
// partials of each halo in chunk order and forms the columns
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
  load_offset_fix<CT>(L.p, pi, H.cfix, H.boxfix, H.frac, f);
  float df[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) df[a] = f32_from_fixcoord(f[a], H.frac);
  return radius_of(df);
}

__device__ __forceinline__ double edge(double r_out, double f, int b, int n) {
  return b == n ? r_out : r_out * pow(f, 1.0 - (double)b / (double)n);
}

// chunk_acc layout per chunk: [0] inner mass (bits of double), [1 + 2b] count,
// [2 + 2b] mass (bits of double)
template <int CT>
__global__ void __launch_bounds__(PT) prof_chunk(ProfileLaunch L) {
  extern __shared__ unsigned char dsm[];
  double* e = (double*)dsm;                        // n_bins + 1 edges
  double* mb = e + (L.n_bins + 1);                 // n_bins masses
  unsigned long long* cb = (unsigned long long*)(mb + L.n_bins);   // n_bins counts
  __shared__ double inner;
  __shared__ unsigned long long cinner;
  __shared__ float r_last;
  const int c = blockIdx.x;
  const int h = L.chunk_halo[c];
  const HaloDev H = L.halos[h];
  const long long start = L.chunk_start[c];
  const long long nb = L.res[h].n_bound;
  const int n = L.n_bins;
  long long* acc = L.chunk_acc + (size_t)c * (1 + 2 * n);
  if (start >= nb) {
    for (int i = threadIdx.x; i < 1 + 2 * n; i += PT) acc[i] = 0;
    return;
  }
  if (threadIdx.x == 0) {
    inner = 0.0;
    cinner = 0ull;
    r_last = L.res[h].r_vir > 0.0 ? 0.0f : bound_radius<CT>(L, H, L.bound_idx[H.offset + nb - 1]);
  }
  for (int b = threadIdx.x; b < n; b += PT) { mb[b] = 0.0; cb[b] = 0ull; }
  __syncthreads();
  const double r_out = L.res[h].r_vir > 0.0 ? L.res[h].r_vir : (double)r_last;
  for (int b = threadIdx.x; b <= n; b += PT) e[b] = edge(r_out, L.r_min_frac, b, n);
  __syncthreads();
  const double lnf = log(L.r_min_frac);
  const long long end = min(nb, start + (long long)PROFILE_CHUNK);
  double my_inner = 0.0;
  unsigned long long my_ci = 0;
  for (long long k = start + threadIdx.x; k < end; k += PT) {
    const long long pi = L.bound_idx[H.offset + k];
    const double r = (double)bound_radius<CT>(L, H, pi);
    const double m = L.p.m ? (CT == AHF_COORD_F64 ? __ldg((const double*)L.p.m + pi)
                                                  : (double)__ldg((const float*)L.p.m + pi))
                           : L.p.m0;
    if (r > e[n]) continue;
    if (r <= e[0]) { my_inner += m; ++my_ci; continue; }
    // first guess from the logarithm, then settle against the FP64 edges
    int b = (int)floor((double)n * (1.0 - log(r / r_out) / lnf));
    b = max(0, min(n - 1, b));
    while (b > 0 && r <= e[b]) --b;
    while (b < n - 1 && r > e[b + 1]) ++b;
    atomicAdd(&cb[b], 1ull);
    if (L.p.m) atomicAdd(&mb[b], m);
  }
  for (int o = 16; o > 0; o >>= 1) my_ci += __shfl_xor_sync(FULL_MASK, my_ci, o);
  if ((threadIdx.x & 31) == 0 && my_ci) atomicAdd(&cinner, my_ci);
  if (L.p.m && my_inner != 0.0) atomicAdd(&inner, my_inner);
  __syncthreads();
  // uniform mass: the inner mass follows exactly from the count
  if (threadIdx.x == 0 && !L.p.m) inner = (double)cinner * L.p.m0;
  __syncthreads();
  if (threadIdx.x == 0) acc[0] = __double_as_longlong(inner);
  for (int b = threadIdx.x; b < n; b += PT) {
    acc[1 + 2 * b] = (long long)cb[b];
    acc[2 + 2 * b] = __double_as_longlong(L.p.m ? mb[b] : (double)cb[b] * L.p.m0);
  }
}

// One CTA per halo: add the chunk partials in chunk order, form the columns.
__global__ void __launch_bounds__(PT) prof_final(ProfileLaunch L, const int* __restrict__ halo_chunk0) {
  const int h = blockIdx.x;
  const int c0 = halo_chunk0[h], c1 = halo_chunk0[h + 1];
  const int n = L.n_bins;
  double* out = L.prof + (size_t)h * n * 4;
  const long long nb = L.res[h].n_bound;
  extern __shared__ unsigned char dsm[];
  double* cnt = (double*)dsm;
  double* mass = cnt + n;
  __shared__ double inner;
  for (int b = threadIdx.x; b < n; b += PT) {
    unsigned long long cc = 0;
    double mm = 0.0;
    for (int c = c0; c < c1; ++c) {
      const long long* acc = L.chunk_acc + (size_t)c * (1 + 2 * n);
      cc += (unsigned long long)acc[1 + 2 * b];
      mm += __longlong_as_double(acc[2 + 2 * b]);
    }
    cnt[b] = (double)cc;
    mass[b] = mm;
  }
  if (threadIdx.x == 0) {
    double in = 0.0;
    for (int c = c0; c < c1; ++c) in += __longlong_as_double(L.chunk_acc[(size_t)c * (1 + 2 * n)]);
    inner = in;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (nb == 0) {
      for (int i = 0; i < 4 * n; ++i) out[i] = 0.0;
      return;
    }
    // r_out as the chunk kernel used it: recompute the outermost radius
    double r_out = L.res[h].r_vir;
    if (!(r_out > 0.0)) {
      const HaloDev H = L.halos[h];
      long long f[3];
      const long long pi = L.bound_idx[H.offset + nb - 1];
      if (L.p.coord_type == AHF_COORD_F64) load_offset_fix<AHF_COORD_F64>(L.p, pi, H.cfix, H.boxfix, H.frac, f);
      else load_offset_fix<AHF_COORD_F32_REL>(L.p, pi, H.cfix, H.boxfix, H.frac, f);
      float df[3];
      for (int a = 0; a < 3; ++a) df[a] = f32_from_fixcoord(f[a], H.frac);
      r_out = (double)radius_of(df);
    }
    double run = inner;
    double lo = edge(r_out, L.r_min_frac, 0, n);
    for (int b = 0; b < n; ++b) {
      const double hi = edge(r_out, L.r_min_frac, b + 1, n);
      run += mass[b];
      out[4 * b + 0] = cnt[b];
      out[4 * b + 1] = run;
      out[4 * b + 2] = mass[b] / (4.0 * M_PI / 3.0 * (hi * hi * hi - lo * lo * lo));
      out[4 * b + 3] = sqrt(L.prm.G * run / hi);
      lo = hi;
    }
  }
}

}  // namespace

int profile_max_bins() { return MAX_BINS; }

cudaError_t launch_profile(const ProfileLaunch& L, const int* halo_chunk0, cudaStream_t s) {
  const size_t sm1 = (size_t)(L.n_bins + 1) * 8 + (size_t)L.n_bins * 16;
  const size_t sm2 = (size_t)L.n_bins * 16;
  cudaError_t e;
  if (L.n_chunks > 0) {
    if (L.p.coord_type == AHF_COORD_F64) {
      e = cudaFuncSetAttribute(prof_chunk<AHF_COORD_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
      if (e != cudaSuccess) return e;
      prof_chunk<AHF_COORD_F64><<<L.n_chunks, PT, sm1, s>>>(L);
    } else {
      e = cudaFuncSetAttribute(prof_chunk<AHF_COORD_F32_REL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
      if (e != cudaSuccess) return e;
      prof_chunk<AHF_COORD_F32_REL><<<L.n_chunks, PT, sm1, s>>>(L);
    }
  }
  e = cudaFuncSetAttribute(prof_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (e != cudaSuccess) return e;
  prof_final<<<L.n_halos, PT, sm2, s>>>(L, halo_chunk0);
  return cudaGetLastError();
}

}  // namespace ahf
