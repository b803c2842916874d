// ms_noalloc.cu -- ms_compress_noalloc: compression into caller memory with no
// device allocation at all.
//
// Some callers of this library cannot call cudaMalloc.  One example is a memory
// manager that wants to compress a buffer while it is serving an allocation
// request and must not re-enter the allocator.  Another is a host that has handed
// every byte of device memory to its own pool up front.  A third is a latency-
// critical path that cannot afford the implicit synchronisation a driver
// allocation may cause.  They get this entry point.  The caller passes the input,
// the output buffer and a two-word result buffer.  The only scratch the kernel
// needs sits in a fixed file-scope device array: the control block, one column
// record and the look-back status words.
//
// That array is shared by every call on a device and keeps the last call's
// contents.  So each call first clears the parts that must start at zero, and
// calls that overlap on the GPU (two streams, or two host threads) race on it.
// Every GPU that loads this library holds the array until the process exits.
#include <algorithm>
#include <mutex>

#include "ms_device.cuh"
#include "ms_kernels.cuh"

namespace ms {
namespace {

constexpr uint64_t kNoallocMaxRows = MS_NOALLOC_MAX_ROWS;
constexpr uint64_t kNoallocTiles = (kNoallocMaxRows + kTile - 1) / kTile;
constexpr size_t kCtlBytes = 256, kMetaBytes = 256;
constexpr size_t kStatusBytes = 8 * (kNoallocTiles + 1);
constexpr size_t kScratchBytes = kCtlBytes + kMetaBytes + kStatusBytes;

// Scratch of ms_compress_noalloc: [DevCtl | DevMeta | look-back status words].
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// Per-device set-up, done once under a once_flag (two host threads making their
// first call on one device at the same time do not race): the array's device
// address, the SM count, the kernel's shared-memory attribute and its occupancy.
struct DeviceSetup {
  std::once_flag once;
  uint8_t* scratch = nullptr;
  int grid_cap = 0;
};
DeviceSetup g_setup[kMaxDevices];
constexpr size_t kProduceSmem = sizeof(typename DirectPlan<OP_COMPRESS>::Smem) * kWarps;

void setup_device(int dev, DeviceSetup* d) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  int sms = 0, occ = 0;
  if (e == cudaSuccess && !p) e = cudaErrorInvalidSymbol;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_produce<OP_COMPRESS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProduceSmem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_produce<OP_COMPRESS>, kThreads, kProduceSmem);
  if (e != cudaSuccess) {
    cudaGetLastError();  // scratch stays null: every call on this device returns MS_ERR_CUDA
    return;
  }
  d->grid_cap = std::max(occ, 1) * std::max(sms, 1);
  d->scratch = static_cast<uint8_t*>(p);
}

// Resets the parts of the scratch that must start at zero and points the control
// block at the caller's output buffer.
__global__ void k_noalloc_prepare(uint8_t* scratch, uint64_t out_ptr, uint64_t out_cap, uint64_t nstatus) {
  DevCtl* ctl = reinterpret_cast<DevCtl*>(scratch);
  uint64_t* status = reinterpret_cast<uint64_t*>(scratch + kCtlBytes + kMetaBytes);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->arena = out_ptr;
    ctl->cap = out_cap;
    ctl->top = 0;
    ctl->high = 0;
    ctl->err = 0;
    ctl->done = 0;
    ctl->err_info = 0;
    ctl->op_n = 0;
    ctl->op_words = 0;
  }
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nstatus;
       i += (uint64_t)gridDim.x * blockDim.x)
    status[i] = 0;
}

// Copies the column size and the device status word into the caller's result.
__global__ void k_noalloc_finish(const uint8_t* scratch, uint64_t* result) {
  const DevCtl* ctl = reinterpret_cast<const DevCtl*>(scratch);
  const DevMeta* meta = reinterpret_cast<const DevMeta*>(scratch + kCtlBytes);
  result[0] = meta->size;
  result[1] = ctl->err;
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" ms_status ms_compress_noalloc(const uint64_t* d_in, uint64_t n, int fmt, int bw, void* d_out,
                                         uint64_t out_cap, uint64_t* d_result, void* stream) {
  static_assert(sizeof(DevCtl) <= kCtlBytes && sizeof(DevMeta) <= kMetaBytes, "scratch layout");
  if ((!d_in && n) || !d_out || !d_result) return MS_ERR_INVALID_ARG;
  if (fmt < MS_UNCOMPR || fmt > MS_FOR_BP || (fmt == MS_STATIC_BP && (bw < 1 || bw > 64)))
    return MS_ERR_INVALID_ARG;
  if (n > kNoallocMaxRows) return MS_ERR_INVALID_ARG;  // beyond the fixed scratch
  if (reinterpret_cast<uintptr_t>(d_in) % 16 || reinterpret_cast<uintptr_t>(d_out) % 16 ||
      reinterpret_cast<uintptr_t>(d_result) % 8)
    return MS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MS_ERR_CUDA;
  // one-time set-up per device, with that device current
  DeviceSetup* d = &g_setup[dev];
  std::call_once(d->once, setup_device, dev, d);
  if (!d->scratch) return MS_ERR_CUDA;
  uint8_t* scratch = d->scratch;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t tiles = std::max<uint64_t>(1, (n + kTile - 1) / kTile);
  k_noalloc_prepare<<<(unsigned)std::min<uint64_t>((tiles + 256) / 256, 64), 256, 0, s>>>(
      scratch, reinterpret_cast<uint64_t>(d_out), out_cap, tiles + 1);
  if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;

  ProduceArgs a{};
  a.ctl = reinterpret_cast<DevCtl*>(scratch);
  a.raw_in = d_in;
  a.raw_n = n;
  a.out_meta = reinterpret_cast<DevMeta*>(scratch + kCtlBytes);
  a.fmt = fmt;
  a.bw = fmt == MS_STATIC_BP ? bw : 0;
  a.status = reinterpret_cast<uint64_t*>(scratch + kCtlBytes + kMetaBytes);
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)d->grid_cap, tiles));
  k_produce<OP_COMPRESS><<<grid, kThreads, kProduceSmem, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
  k_noalloc_finish<<<1, 1, 0, s>>>(scratch, d_result);
  return cudaGetLastError() == cudaSuccess ? MS_OK : MS_ERR_CUDA;
}
