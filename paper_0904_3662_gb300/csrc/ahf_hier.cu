// Hosts and subhaloes in dependency order (Sect. 2.1): the kernels around
// each level's unbinding.
//
// A level is unbound with member lists that leave out the candidates a
// descendant already bound: `owner` holds, per particle, the last halo that
// bound it (level rank in the high 32 bits, halo index in the low 32, so an
// atomic maximum keeps the latest level and, within a level, the highest
// index); `anc` maps every deeper halo to its ancestor on the current level.
// The level's results land in scratch (records by level position, removal
// iterations by compacted slot) and are scattered to the caller's arrays.
#include <cstdint>

#include "ahf_device.cuh"

namespace ahf {
namespace {

constexpr int PT = 256;

// One CTA per halo of the level: the kept candidates, compacted in slot order.
__global__ void __launch_bounds__(PT) hier_compact(HierLaunch L) {
  __shared__ long long base;
  __shared__ int wsum[PT / 32];
  const int i = blockIdx.x;
  const int h = L.level[i];
  const long long off = L.halos[h].offset, cnt = L.halos[h].count;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (long long s0 = 0; s0 < cnt; s0 += PT) {
    const long long j = s0 + threadIdx.x;
    long long q = -1;
    bool keep = false;
    if (j < cnt) {
      const long long slot = off + j;
      q = L.member_idx ? L.member_idx[slot] : slot;
      if (q >= 0 && q < L.n_particles) {
        const long long own = L.owner[q];
        const int t = own >= 0 ? (int)(own & 0xffffffffll) : -1;
        keep = !(t >= 0 && L.anc[t] == h);
      } else {
        keep = true;              // left to the unbinding, which reports the bad index
      }
    }
    const unsigned b = __ballot_sync(FULL_MASK, keep);
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < PT / 32; ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (keep) {
      const long long pos = base + before + __popc(b & lanemask_lt());
      L.members[off + pos] = q;
      L.cand_map[off + pos] = off + j;
    }
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) L.kept[i] = base;
}

// One CTA per halo of the level: its record, its removal iterations by
// candidate slot, and the owner marks of its bound particles.
__global__ void __launch_bounds__(PT) hier_scatter(HierLaunch L) {
  const int i = blockIdx.x;
  const int h = L.level[i];
  const long long off = L.halos[h].offset, cnt = L.halos[h].count;
  const ahf_result r = L.res_level[i];
  if (threadIdx.x == 0) L.res[h] = r;
  if (L.removed_iter) {
    for (long long j = threadIdx.x; j < cnt; j += PT) L.removed_iter[off + j] = -1;
    __syncthreads();
    const long long kept = L.kept[i];
    for (long long j = threadIdx.x; j < kept; j += PT) L.removed_iter[L.cand_map[off + j]] = L.rem_level[off + j];
  }
  const long long tag = ((long long)L.rank << 32) | (long long)h;
  for (long long k = threadIdx.x; k < r.n_bound; k += PT) {
    const long long q = L.bound_idx[off + k];
    if (q >= 0 && q < L.n_particles) atomicMax((long long*)&L.owner[q], tag);
  }
}

}  // namespace

cudaError_t launch_hier_compact(const HierLaunch& L, int n_level, cudaStream_t s) {
  if (n_level > 0) hier_compact<<<n_level, PT, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_hier_scatter(const HierLaunch& L, int n_level, cudaStream_t s) {
  if (n_level > 0) hier_scatter<<<n_level, PT, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace ahf
