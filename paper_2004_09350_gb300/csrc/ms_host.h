// ms_host.h -- host-side context and column structures of libms.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "morphstore.h"
#include "ms_device.cuh"

struct ms_column {
  ms_ctx* ctx;
  int slot;         // metadata slot on the device
  int fmt, bw;      // format (host-known)
  uint64_t n_max;   // host-known upper bound on the length
  bool arena;       // carved from the arena (else allocated by the callbacks)
  bool freed;       // released by the caller, waiting for LIFO reclamation
  void* ext;        // external buffer (non-arena columns)
};

struct ms_prof_rec {
  int kernel;
  cudaEvent_t start, stop;
};

struct ms_ctx {
  int device = 0, sms = 0;
  ms_alloc_fn alloc = nullptr;
  ms_free_fn free_fn = nullptr;
  void* user = nullptr;
  uint8_t* arena = nullptr;
  uint64_t arena_cap = 0;
  ms::DevCtl* ctl = nullptr;
  ms::DevMeta* metas = nullptr;
  std::vector<int> free_slots;
  std::vector<ms_column*> stack;  // arena columns in allocation order
  std::vector<ms_column*> live;
  uint8_t* work = nullptr;
  uint64_t work_cap = 0;
  uint64_t* pin = nullptr;  // pinned host scratch
  uint64_t last_err_info = 0;
  bool prof_on = false;
  std::vector<ms_prof_rec> prof;
  std::vector<cudaEvent_t> event_pool;
};

namespace ms {

inline uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline uint64_t align_up(uint64_t a, uint64_t b) { return cdiv(a, b) * b; }

void* dev_alloc(ms_ctx* c, size_t bytes);
void dev_free(ms_ctx* c, void* p);
ms_status cuda_status(cudaError_t e);
bool valid_format(int fmt, int bw);
// Block-format outputs (headers + payloads; placed after staging), and the layout a
// format is read as (FOR / DELTA cascaded with static BP use the FOR+BP / DELTA+BP layout).
inline bool host_block_fmt(int f) {
  return f == MS_DYN_BP || f == MS_DELTA_BP || f == MS_FOR_BP || f == MS_FOR_STATIC_BP || f == MS_DELTA_STATIC_BP;
}
inline int host_layout_fmt(int f) {
  return f == MS_FOR_STATIC_BP ? MS_FOR_BP : (f == MS_DELTA_STATIC_BP ? MS_DELTA_BP : f);
}
// formats with a caller-chosen width (static_bw in 1..64)
inline bool has_static_bw(int f) { return f == MS_STATIC_BP || f == MS_FOR_STATIC_BP || f == MS_DELTA_STATIC_BP; }
int take_slot(ms_ctx* c);
ms_column* new_arena_column(ms_ctx* c, int fmt, int bw, uint64_t n_max);
void drop_new_column(ms_ctx* c, ms_column* col);
// Makes sure the scratch area holds at least `bytes`; synchronises when it grows.
ms_status ensure_work(ms_ctx* c, uint64_t bytes);

// An NVTX range around one entry point (visible to nsys and to ncu's --nvtx filters;
// a no-op without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define MS_TRACE() ::ms::NvtxRange ms_trace_range_(__func__)

// Brackets one kernel launch with profiling events when profiling is on.
class ProfScope {
 public:
  ProfScope(ms_ctx* c, int kernel, cudaStream_t s);
  ~ProfScope();

 private:
  ms_ctx* c_;
  cudaStream_t s_;
  int idx_ = -1;
};

}  // namespace ms
