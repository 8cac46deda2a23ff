// Launch layer shared by single-instance and batched execution.
//
// Every kernel of the solve path is written once as a block body `K::body(args, blk, nblk)`
// (blk = the block's index in the instance's own grid, nblk = that grid's size) and reached
// through two entry points:
//   k_one<K>   one instance, args in the parameter space, grid = nblk blocks;
//   k_many<K>  many instances in one launch: block b runs work[b] = (args row, blk, nblk, slot)
//              with the args row read from a device table.  Blocks of a slot whose entry in
//              `active` is 0 return at once (the slot left the batch).
// Both entry points are launched with programmatic stream serialization (programmatic dependent
// launch): a kernel may be scheduled while its predecessor in the stream is still running, and
// its first instruction, griddepcontrol.wait, holds every thread until the predecessor grid has
// completed and its memory is visible.  No block touches memory before that wait, so the order of
// the launches is preserved; only the launch latency overlaps the predecessor's tail.  (Without
// the launch attribute the wait returns at once.)  The blocks do not signal their dependents early
// (griddepcontrol.launch_dependents): measured on the channel solve, successor blocks parked at
// their wait on the SMs slowed it down (49.9 against 49.05 ms).
// submit<K>() launches k_one immediately, or, while a Recorder is installed on the calling
// thread, appends (kernel, args, nblk, shared bytes) to it instead.  The batching engine records
// the same host code for every instance and merges the recordings step by step into k_many
// launches, so a batched instance runs exactly the arithmetic of its single-instance solve.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <vector>

namespace gs {

cudaError_t launched(cudaError_t e, int kernels);

struct WorkItem {
  int arg;   // row of the argument table
  int blk;   // block index within the instance's grid
  int nblk;  // the instance's grid size
  int slot;  // engine slot (-1: not maskable)
};

using BatchFn = cudaError_t (*)(const void* tab, const WorkItem* work, int nwork, const int* active, size_t smem,
                                cudaStream_t st);

struct RecOp {
  BatchFn fn;
  int nblk;
  int arg_size;
  size_t arg_off;  // offset of the argument bytes in Recorder::bytes
  size_t smem;
};

struct Recorder {
  std::vector<RecOp> ops;
  std::vector<unsigned char> bytes;
  void add(BatchFn fn, const void* args, int size, int nblk, size_t smem) {
    const size_t off = (bytes.size() + 15) & ~size_t(15);
    bytes.resize(off + size);
    std::memcpy(bytes.data() + off, args, size);
    ops.push_back(RecOp{fn, nblk, size, off, smem});
  }
  void clear() {
    ops.clear();
    bytes.clear();
  }
};

// recorder installed on this thread (nullptr: launch immediately)
Recorder*& current_recorder();

// Raise a kernel's dynamic shared memory limit to at least smem bytes on the current device.  The
// attribute is per device, so the largest size enabled so far is kept per (kernel, device); the
// counters are atomics because contexts are built on several host threads at once.
constexpr int kMaxDevices = 64;
template <class F>
cudaError_t ensure_dynamic_smem(F* fn, size_t smem, std::atomic<size_t>* enabled) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (enabled[dev].load(std::memory_order_acquire) >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  size_t cur = enabled[dev].load(std::memory_order_relaxed);
  while (cur < smem && !enabled[dev].compare_exchange_weak(cur, smem, std::memory_order_acq_rel)) {
  }
  return cudaSuccess;
}

__device__ __forceinline__ void wait_prerequisite_grids() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class K>
__global__ void __launch_bounds__(K::THREADS, K::MINB) k_one(const typename K::Args a) {
  wait_prerequisite_grids();
  K::body(a, (int)blockIdx.x, (int)gridDim.x);
}

template <class K>
__global__ void __launch_bounds__(K::THREADS, K::MINB)
    k_many(const typename K::Args* __restrict__ tab, const WorkItem* __restrict__ work, const int* __restrict__ active) {
  wait_prerequisite_grids();
  const WorkItem w = work[blockIdx.x];
  if (active != nullptr && w.slot >= 0 && active[w.slot] == 0) return;
  K::body(tab[w.arg], w.blk, w.nblk);
}

template <class K>
cudaError_t batch_launch(const void* tab, const WorkItem* work, int nwork, const int* active, size_t smem,
                         cudaStream_t st) {
  if (nwork <= 0) return cudaSuccess;
  static std::atomic<size_t> enabled[kMaxDevices];  // zero-initialised (static storage)
  cudaError_t e = ensure_dynamic_smem(k_many<K>, smem, enabled);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)nwork);
  cfg.blockDim = dim3(K::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return launched(cudaLaunchKernelEx(&cfg, k_many<K>, (const typename K::Args*)tab, work, active), 1);
}

template <class K>
cudaError_t submit(const typename K::Args& a, long long nblk, size_t smem, cudaStream_t st) {
  if (nblk < 1) nblk = 1;
  if (Recorder* r = current_recorder()) {
    r->add(&batch_launch<K>, &a, (int)sizeof(a), (int)nblk, smem);
    return cudaSuccess;
  }
  static std::atomic<size_t> enabled[kMaxDevices];
  cudaError_t e = ensure_dynamic_smem(k_one<K>, smem, enabled);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)nblk);
  cfg.blockDim = dim3(K::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return launched(cudaLaunchKernelEx(&cfg, k_one<K>, a), 1);
}

}  // namespace gs
