// Launcher of the 2D strip kernel (gs_strip2d.cuh).
#include <atomic>

#include "gs_strip2d.cuh"

namespace gs {
namespace {

int device_index() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
  return dev;
}

int sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  const int dev = device_index();
  if (dev >= 0 && cache[dev].load(std::memory_order_relaxed) > 0) return cache[dev].load(std::memory_order_relaxed);
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev) != cudaSuccess || v <= 0) v = 1;
  if (dev >= 0) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Resident CTAs per SM of the kernel with `smem` bytes of dynamic shared memory (per device).
template <class K>
int ctas_per_sm(size_t smem) {
  static std::atomic<size_t> enabled[kMaxDevices];
  static std::atomic<int> cache[kMaxDevices];
  const int dev = device_index();
  if (dev >= 0 && cache[dev].load(std::memory_order_relaxed) > 0) return cache[dev].load(std::memory_order_relaxed);
  int n = 1;
  if (ensure_dynamic_smem(k_one<K>, smem, enabled) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_one<K>, K::THREADS, smem) == cudaSuccess && n > 0) {
    if (dev >= 0) cache[dev].store(n, std::memory_order_relaxed);
  } else {
    cudaGetLastError();
    n = 1;
  }
  return n;
}

// Batches per segment: minimise (waves of the grid) x (batches per CTA), then the rows evaluated.
void choose_segments(int n0, int n1, int slots, int* strips, int* segs, int* nb_out) {
  const int s = (n0 + strip2d::OC - 1) / strip2d::OC;
  const int nb_max = (n1 + 1 + strip2d::NW - 1) / strip2d::NW;
  long long best_cost = -1, best_rows = 0;
  int best = 1;
  for (int nb = 1; nb <= nb_max; ++nb) {
    const int R = strip2d::NW * nb - 1;
    const long long grid = (long long)s * ((n1 + R - 1) / R);
    const long long waves = (grid + slots - 1) / slots;
    const long long cost = waves * nb;
    const long long rows = grid * nb;
    if (best_cost < 0 || cost < best_cost || (cost == best_cost && rows < best_rows)) {
      best_cost = cost;
      best_rows = rows;
      best = nb;
    }
  }
  const int R = strip2d::NW * best - 1;
  *strips = s;
  *segs = (n1 + R - 1) / R;
  *nb_out = best;
}

template <typename T, int MODE>
cudaError_t launch_mode(TileArgs<T> a, cudaStream_t st) {
  using K = strip2d::Strip2dK<T, MODE>;
  const size_t smem = strip2d::Smem<T, MODE>::BYTES;
  const int slots = sm_count() * ctas_per_sm<K>(smem);
  int strips, segs, nb;
  choose_segments(a.g.n[0], a.g.n[1], slots, &strips, &segs, &nb);
  a.tiles[0] = strips;
  a.tiles[1] = segs;
  a.tiles[2] = nb;
  return submit<K>(a, (long long)strips * segs, smem, st);
}

}  // namespace

template <typename T>
cudaError_t launch_strip2d(int mode, TileArgs<T> a, cudaStream_t st) {
  if (a.g.dim != 2) return cudaErrorInvalidValue;
  if (mode == TILE_APPLY) return launch_mode<T, TILE_APPLY>(a, st);
  if (mode == TILE_RESID) return launch_mode<T, TILE_RESID>(a, st);
  return launch_mode<T, TILE_CHEB>(a, st);
}
template cudaError_t launch_strip2d<float>(int, TileArgs<float>, cudaStream_t);
template cudaError_t launch_strip2d<double>(int, TileArgs<double>, cudaStream_t);

// Fault-path probe: waits on a phase of an mbarrier that nothing completes (count 1, no arrival),
// through the same bounded wait as the strip kernel, which gives up and sets *err.
__global__ void k_wait_probe(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) strip2d::mbar_init(&bar, 1);
  __syncthreads();
  strip2d::mbar_wait(&bar, 0u, err);
}
cudaError_t launch_wait_probe(int* err, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(err);
  return launched(cudaGetLastError(), 1);
}

}  // namespace gs
