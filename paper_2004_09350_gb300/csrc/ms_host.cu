// ms_host.cu -- context, arena, column management and error reporting of libms.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "ms_host.h"

namespace ms {

static int g_last_cuda_error = 0;  // last failing cudaError_t seen by the library

ms_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MS_OK;
  g_last_cuda_error = (int)e;
  return MS_ERR_CUDA;
}

void* dev_alloc(ms_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (c->alloc) return c->alloc(bytes, c->user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(ms_ctx* c, void* p) {
  if (!p) return;
  if (c->free_fn) c->free_fn(p, c->user);
  else cudaFree(p);
}

bool valid_format(int fmt, int bw) {
  if (fmt < MS_UNCOMPR || fmt > MS_DELTA_STATIC_BP) return false;
  if (has_static_bw(fmt) && (bw < 1 || bw > 64)) return false;
  return true;
}

int take_slot(ms_ctx* c) {
  if (c->free_slots.empty()) return -1;
  int s = c->free_slots.back();
  c->free_slots.pop_back();
  return s;
}

ms_column* new_arena_column(ms_ctx* c, int fmt, int bw, uint64_t n_max) {
  int slot = take_slot(c);
  if (slot < 0) return nullptr;
  ms_column* col = new (std::nothrow) ms_column;
  if (!col) {
    c->free_slots.push_back(slot);
    return nullptr;
  }
  col->ctx = c;
  col->slot = slot;
  col->fmt = fmt;
  col->bw = has_static_bw(fmt) ? bw : 0;
  col->n_max = n_max;
  col->arena = true;
  col->freed = false;
  col->ext = nullptr;
  c->stack.push_back(col);
  c->live.push_back(col);
  return col;
}

void drop_new_column(ms_ctx* c, ms_column* col) {
  // only valid for a column whose kernel was never enqueued
  c->stack.erase(std::remove(c->stack.begin(), c->stack.end(), col), c->stack.end());
  c->live.erase(std::remove(c->live.begin(), c->live.end(), col), c->live.end());
  c->free_slots.push_back(col->slot);
  delete col;
}

ms_status ensure_work(ms_ctx* c, uint64_t bytes) {
  if (bytes <= c->work_cap) return MS_OK;
  if (cuda_status(cudaDeviceSynchronize()) != MS_OK) return MS_ERR_CUDA;
  dev_free(c, c->work);
  const uint64_t cap = bytes;  // exactly what the longest column asks for: no slack
  c->work = static_cast<uint8_t*>(dev_alloc(c, cap));
  if (!c->work) {
    c->work_cap = 0;
    return MS_ERR_NOMEM;
  }
  c->work_cap = cap;
  return MS_OK;
}

static cudaEvent_t pooled_event(ms_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

ProfScope::ProfScope(ms_ctx* c, int kernel, cudaStream_t s) : c_(c), s_(s) {
  if (!c->prof_on) return;
  ms_prof_rec r{kernel, pooled_event(c), pooled_event(c)};
  if (!r.start || !r.stop) return;
  cudaEventRecord(r.start, s);
  c->prof.push_back(r);
  idx_ = (int)c->prof.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx_ >= 0) cudaEventRecord(c_->prof[idx_].stop, s_);
}

__global__ void k_write_meta(DevMeta* m, DevMeta v) { *m = v; }

__global__ void k_set_top(DevCtl* ctl, const DevMeta* m) {
  ctl->top = m->ptr - ctl->arena;
}

// Checks the header chain of an imported block-format column (Sec. 4.1 layout).
__global__ void k_validate(DevMeta* m, DevCtl* ctl) {
  const uint64_t nb = m->nb;
  const uint64_t* h = reinterpret_cast<const uint64_t*>(m->ptr);
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nb;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t w0 = h[2 * k];
    const uint64_t b = w0 & 255, off = w0 >> 8;
    bool ok = b <= 64;
    if (k == 0) ok = ok && off == 0;
    if (k + 1 < nb) ok = ok && (h[2 * (k + 1)] >> 8) == off + 8 * b;
    if (k + 1 == nb) {
      ok = ok && 16 * nb + 8 * (off + 8 * b) + 8 * (m->n % kBlock) <= m->size;
      m->pwords = off + 8 * b;  // the payload ends behind the last block
    }
    if (!ok) set_error(ctl, MS_ERR_FORMAT, k);
  }
  if (nb == 0 && blockIdx.x == 0 && threadIdx.x == 0 && 8 * (m->n % kBlock) > m->size)
    set_error(ctl, MS_ERR_FORMAT, 0);
}

}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_ctx_create(ms_ctx** out, int device, uint64_t arena_bytes, uint64_t max_rows,
                        ms_alloc_fn alloc, ms_free_fn free_fn, void* user) {
  if (!out) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (free_fn == nullptr)) return MS_ERR_INVALID_ARG;
  if (cuda_status(cudaSetDevice(device)) != MS_OK) return MS_ERR_CUDA;
  ms_ctx* c = new (std::nothrow) ms_ctx;
  if (!c) return MS_ERR_NOMEM;
  c->device = device;
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  arena_bytes = align_up(std::max<uint64_t>(arena_bytes, 1 << 20), 256);
  c->arena = static_cast<uint8_t*>(dev_alloc(c, arena_bytes));
  c->ctl = static_cast<DevCtl*>(dev_alloc(c, sizeof(DevCtl)));
  c->metas = static_cast<DevMeta*>(dev_alloc(c, sizeof(DevMeta) * kMaxSlots));
  if (cudaHostAlloc(&c->pin, 4096, cudaHostAllocDefault) != cudaSuccess) c->pin = nullptr;
  if (!c->arena || !c->ctl || !c->metas || !c->pin) {
    ms_ctx_destroy(c);
    return MS_ERR_NOMEM;
  }
  c->arena_cap = arena_bytes;
  DevCtl h{};
  h.arena = reinterpret_cast<uint64_t>(c->arena);
  h.cap = arena_bytes;
  if (cudaMemcpy(c->ctl, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->metas, 0, sizeof(DevMeta) * kMaxSlots) != cudaSuccess) {
    ms_ctx_destroy(c);
    return MS_ERR_CUDA;
  }
  c->free_slots.reserve(kMaxSlots);
  for (int s = kMaxSlots - 1; s >= 0; s--) c->free_slots.push_back(s);
  uint64_t nch = cdiv(std::max<uint64_t>(max_rows, 1), kBlock);
  ms_status st = ensure_work(c, 128 * nch + 4096);
  if (st != MS_OK) {
    ms_ctx_destroy(c);
    return st;
  }
  *out = c;
  return MS_OK;
}

ms_status ms_ctx_destroy(ms_ctx* c) {
  if (!c) return MS_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (ms_column* col : c->live) {
    if (!col->arena) dev_free(c, col->ext);
    delete col;
  }
  c->live.clear();
  dev_free(c, c->work);
  dev_free(c, c->arena);
  dev_free(c, c->ctl);
  dev_free(c, c->metas);
  if (c->pin) cudaFreeHost(c->pin);
  for (auto& r : c->prof) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  delete c;
  return MS_OK;
}

ms_status ms_get_error(ms_ctx* c, void* stream) {
  if (!c) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(c->pin, &c->ctl->err, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    return MS_ERR_CUDA;
  }
  uint32_t err = static_cast<uint32_t>(c->pin[0] & 0xffffffffu);
  c->last_err_info = c->pin[1];
  if (err != 0) {
    // clear the error and release a stage that a failed producer may have left taken
    uint32_t zero = 0;
    if (cuda_status(cudaMemcpy(&c->ctl->err, &zero, 4, cudaMemcpyHostToDevice)) != MS_OK ||
        cuda_status(cudaMemset(&c->ctl->stage, 0, 8)) != MS_OK)
      return MS_ERR_CUDA;
  }
  return static_cast<ms_status>(err);
}

uint64_t ms_last_error_info(ms_ctx* c) { return c ? c->last_err_info : 0; }

uint64_t ms_work_bytes(const ms_ctx* c) { return c ? c->work_cap : 0; }

ms_status ms_arena_usage(ms_ctx* c, uint64_t* in_use, uint64_t* high, void* stream) {
  if (!c) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(c->pin, &c->ctl->top, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MS_ERR_CUDA;
  if (in_use) *in_use = c->pin[0];
  if (high) *high = c->pin[1];
  return MS_OK;
}

ms_status ms_arena_reset_high_water(ms_ctx* c, void* stream) {
  if (!c) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return cuda_status(cudaMemcpyAsync(&c->ctl->high, &c->ctl->top, 8, cudaMemcpyDeviceToDevice, s));
}

ms_status ms_column_import(ms_ctx* c, int fmt, int bw, uint64_t n, const void* src, uint64_t size,
                           ms_column** out, void* stream) {
  if (!c || !out || (!src && size)) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_format(fmt, bw)) return MS_ERR_INVALID_ARG;
  const bool blockfmt = host_block_fmt(fmt);
  uint64_t nb = blockfmt ? n / kBlock : 0;
  if (fmt == MS_UNCOMPR && size < 8 * n) return MS_ERR_FORMAT;
  if (fmt == MS_STATIC_BP && size < 8 * cdiv(n * (uint64_t)bw, 64)) return MS_ERR_FORMAT;
  if (blockfmt && size < 16 * nb + 8 * (n % kBlock)) return MS_ERR_FORMAT;
  if (fmt == MS_RLE) {  // R runs and the directory: size = 16 R + 8 ceil(n / 512)
    const uint64_t dir = 8 * cdiv(n, kBlock);
    if (size < dir || (size - dir) % 16) return MS_ERR_FORMAT;
    nb = (size - dir) / 16;
    if ((n == 0) != (nb == 0) || nb > n) return MS_ERR_FORMAT;
  }
  int slot = take_slot(c);
  if (slot < 0) return MS_ERR_NOMEM;
  void* buf = dev_alloc(c, align_up(size + 64, 256));
  if (!buf) {
    c->free_slots.push_back(slot);
    return MS_ERR_NOMEM;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = size ? cudaMemcpyAsync(buf, src, size, cudaMemcpyDefault, s) : cudaSuccess;
  DevMeta m{};
  m.n = n;
  m.ptr = reinterpret_cast<uint64_t>(buf);
  m.size = size;
  m.nb = nb;
  m.fmt = static_cast<uint32_t>(fmt);
  m.bw = has_static_bw(fmt) ? static_cast<uint32_t>(bw) : 0;
  m.pwords = 0;  // block formats: set by the validation kernel from the last header
  if (e == cudaSuccess) {
    ProfScope ps(c, MS_K_ARENA, s);
    k_write_meta<<<1, 1, 0, s>>>(c->metas + slot, m);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && blockfmt) {
    ProfScope ps(c, MS_K_VALIDATE, s);
    k_validate<<<(unsigned)std::min<uint64_t>(cdiv(std::max<uint64_t>(nb, 1), 256), 1024), 256, 0, s>>>(
        c->metas + slot, c->ctl);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    dev_free(c, buf);
    c->free_slots.push_back(slot);
    return MS_ERR_CUDA;
  }
  ms_column* col = new (std::nothrow) ms_column;
  if (!col) {
    cudaStreamSynchronize(s);
    dev_free(c, buf);
    c->free_slots.push_back(slot);
    return MS_ERR_NOMEM;
  }
  col->ctx = c;
  col->slot = slot;
  col->fmt = fmt;
  col->bw = has_static_bw(fmt) ? bw : 0;
  col->n_max = n;
  col->arena = false;
  col->freed = false;
  col->ext = buf;
  c->live.push_back(col);
  *out = col;
  return MS_OK;
}

ms_status ms_column_info(ms_ctx* c, const ms_column* col, ms_column_meta* out, void* stream) {
  if (!c || !col || !out || col->ctx != c) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(c->pin, c->metas + col->slot, sizeof(DevMeta), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MS_ERR_CUDA;
  DevMeta m;
  memcpy(&m, c->pin, sizeof m);
  out->n = m.n;
  out->fmt = static_cast<int32_t>(m.fmt);
  out->static_bw = static_cast<int32_t>(m.bw);
  out->size_bytes = m.size;
  out->n_blocks = m.nb;
  out->payload_words = m.pwords;
  out->device_ptr = m.ptr;
  return MS_OK;
}

uint64_t ms_column_max_rows(const ms_column* col) { return col ? col->n_max : 0; }

ms_status ms_column_export(ms_ctx* c, const ms_column* col, void* dst, uint64_t cap, uint64_t* size_out,
                           void* stream) {
  ms_column_meta m;
  ms_status st = ms_column_info(c, col, &m, stream);
  if (st != MS_OK) return st;
  if (size_out) *size_out = m.size_bytes;
  if (m.size_bytes > cap || (!dst && m.size_bytes)) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (m.size_bytes &&
      (cudaMemcpyAsync(dst, reinterpret_cast<const void*>(m.device_ptr), m.size_bytes, cudaMemcpyDefault, s) !=
           cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    return MS_ERR_CUDA;
  return MS_OK;
}

ms_status ms_column_free(ms_ctx* c, ms_column* col, void* stream) {
  if (!c || !col || col->ctx != c || col->freed) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!col->arena) {
    // the buffer may still be read by enqueued work: drain the stream first
    if (cuda_status(cudaStreamSynchronize(s)) != MS_OK) return MS_ERR_CUDA;
    dev_free(c, col->ext);
    c->free_slots.push_back(col->slot);
    c->live.erase(std::remove(c->live.begin(), c->live.end(), col), c->live.end());
    delete col;
    return MS_OK;
  }
  col->freed = true;
  int lowest = -1;
  while (!c->stack.empty() && c->stack.back()->freed) {
    ms_column* t = c->stack.back();
    c->stack.pop_back();
    lowest = t->slot;
    c->live.erase(std::remove(c->live.begin(), c->live.end(), t), c->live.end());
    c->free_slots.push_back(t->slot);
    delete t;
  }
  if (lowest >= 0) {
    // the arena top returns to the start of the lowest popped column; the slot's
    // metadata is read by the kernel before any later kernel can reuse the slot
    ProfScope ps(c, MS_K_ARENA, s);
    k_set_top<<<1, 1, 0, s>>>(c->ctl, c->metas + lowest);
    if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
  }
  return MS_OK;
}

ms_status ms_profile_enable(ms_ctx* c, int on) {
  if (!c) return MS_ERR_INVALID_ARG;
  c->prof_on = on != 0;
  return MS_OK;
}

ms_status ms_profile_collect(ms_ctx* c, ms_kernel_time* out, int max, int* n_out) {
  if (!c || (!out && max > 0)) return MS_ERR_INVALID_ARG;
  if (cuda_status(cudaDeviceSynchronize()) != MS_OK) return MS_ERR_CUDA;
  ms_kernel_time acc[MS_K_COUNT];
  for (int k = 0; k < MS_K_COUNT; k++) acc[k] = ms_kernel_time{k, 0, 0.0};
  for (auto& r : c->prof) {
    float ms = 0.f;
    if (r.kernel >= 0 && r.kernel < MS_K_COUNT && cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      acc[r.kernel].launches++;
      acc[r.kernel].total_ms += ms;
    }
    c->event_pool.push_back(r.start);
    c->event_pool.push_back(r.stop);
  }
  c->prof.clear();
  int n = 0;
  for (int k = 0; k < MS_K_COUNT && n < max; k++)
    if (acc[k].launches) out[n++] = acc[k];
  if (n_out) *n_out = n;
  return MS_OK;
}

const char* ms_kernel_name(int k) {
  static const char* names[MS_K_COUNT] = {"mark",       "emit",     "compress", "decompress",    "project",
                                          "calc",       "agg_sum",  "group_sum", "build_keys",   "validate",
                                          "scan",       "place",    "stats",     "batch",        "select_packed",
                                          "arena",      "rle"};
  return (k >= 0 && k < MS_K_COUNT) ? names[k] : "?";
}

int ms_last_cuda_error(void) { return g_last_cuda_error; }

const char* ms_cuda_error_string(int code) { return cudaGetErrorString((cudaError_t)code); }

}  // extern "C"
