// Device runtime of the hierarchical collective engine: upload of the
// memoized plan (paper Sec. 5.2), the persistent sm_103a executor kernel, and
// the non-blocking start / blocking wait of the C ABI (Sec. 3.3, Listing 2).
//
// Executor design.  One launch executes the whole step table.  Work items
// (runs of step segments that share one pipeline slot, so that no item waits
// on itself) are claimed in table order from a global ticket; an item only
// waits for steps of earlier items, all of which were claimed by CTAs that
// are already running, so the launch makes progress for any grid size.  A
// step's predecessors signal it with release adds on its dependency counter;
// the item's CTA polls the counters with acquire loads, bounded by a time
// limit after which the launch aborts and reports HICCL_ERR_TIMEOUT.  Within
// an item every warp moves whole 4 KiB segments with 16-byte vector loads
// (L2-cached, not L1: the data may have been written by another SM in this
// launch) and stores; a copy reads its source once and writes every
// destination; a reduce folds its inputs in the fixed order in FP32 (or int32)
// without fused multiply-add.  Counters accumulate over launches: the targets
// of launch e are e times the per-launch counts, so no reset kernel runs
// between starts.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "hiccl_internal.h"

namespace hiccl {


struct DevState {
  int device = -1;
  int nsm = 0;
  int occ[4] = {0, 0, 0, 0};        // resident CTAs per SM for 64/128/256/512 threads
  void *table = nullptr;            // read-only arrays
  void *counters = nullptr;         // dep[], done[], ctl
  size_t counters_bytes = 0;
  void *scratch = nullptr;
  unsigned long long *host_err = nullptr;
  unsigned long long *host_err_dev = nullptr;
  cudaEvent_t done_ev = nullptr;
  DevTable t{};
  std::vector<uint32_t> indeg;      // host copy, for fault injection
  uint32_t *indeg_dev = nullptr;
};

// ---------------------------------------------------------------------------
// memory-model helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_acq_rel_add(unsigned long long *p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void raise_error(const DevTable &T, unsigned long long code) {
  if (atomicCAS(&T.ctl->err, 0ull, code) == 0ull) *(volatile unsigned long long *)T.host_err = code;
}

// ---------------------------------------------------------------------------
// data movement of one segment by one warp
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T ldg_ro(const T *p) { return __ldg(p); }

__device__ __forceinline__ uint4 ld16(const char *p) { return __ldcg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ void st16(char *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

__device__ __forceinline__ uint4 add4(uint4 a, uint4 b, uint32_t dt) {
  if (dt == HICCL_F32) {
    a.x = __float_as_uint(__fadd_rn(__uint_as_float(a.x), __uint_as_float(b.x)));
    a.y = __float_as_uint(__fadd_rn(__uint_as_float(a.y), __uint_as_float(b.y)));
    a.z = __float_as_uint(__fadd_rn(__uint_as_float(a.z), __uint_as_float(b.z)));
    a.w = __float_as_uint(__fadd_rn(__uint_as_float(a.w), __uint_as_float(b.w)));
  } else {   // int32, wrapping
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
  }
  return a;
}

// copy bytes [lo, lo + n) of the source to every destination (n <= SEG_BYTES)
__device__ __forceinline__ void warp_copy(const unsigned long long *ptrs, uint32_t ndst, unsigned long long lo,
                                          uint32_t n, bool aligned, int lane) {
  const char *src = reinterpret_cast<const char *>(ptrs[0]) + lo;
  uint32_t done = 0;
  if (aligned) {
    constexpr int U = SEG_BYTES / (16 * 32);   // one pass covers the segment
    const uint32_t nvec = n >> 4;
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = u * 32 + lane;
      if (i < nvec) v[u] = ld16(src + (i << 4));
    }
    for (uint32_t k = 0; k < ndst; ++k) {
      char *dst = reinterpret_cast<char *>(ptrs[1 + k]) + lo;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = u * 32 + lane;
        if (i < nvec) st16(dst + (i << 4), v[u]);
      }
    }
    done = nvec << 4;
  }
  for (uint32_t b = done + lane; b < n; b += 32) {
    const char v = __ldcg(src + b);
    for (uint32_t k = 0; k < ndst; ++k) (reinterpret_cast<char *>(ptrs[1 + k]) + lo)[b] = v;
  }
}

// out[lo, lo + n) = in_0 + in_1 + ... (left fold, fixed order; n <= SEG_BYTES)
__device__ __forceinline__ void warp_reduce(const unsigned long long *ptrs, uint32_t nsrc, uint32_t dt,
                                            unsigned long long lo, uint32_t n, bool aligned, int lane) {
  char *dst = reinterpret_cast<char *>(ptrs[nsrc]) + lo;
  uint32_t done = 0;
  if (aligned) {
    constexpr int U = 4;
    const uint32_t nvec = n >> 4;
    for (uint32_t base = 0; base < nvec; base += 32 * U) {
      uint4 acc[U];
      const char *s0 = reinterpret_cast<const char *>(ptrs[0]) + lo;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = base + u * 32 + lane;
        if (i < nvec) acc[u] = ld16(s0 + (i << 4));
      }
      for (uint32_t q = 1; q < nsrc; ++q) {
        const char *sq = reinterpret_cast<const char *>(ptrs[q]) + lo;
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t i = base + u * 32 + lane;
          if (i < nvec) v[u] = ld16(sq + (i << 4));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = add4(acc[u], v[u], dt);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = base + u * 32 + lane;
        if (i < nvec) st16(dst + (i << 4), acc[u]);
      }
    }
    done = nvec << 4;
  }
  // element tail (or the whole unaligned range): 4-byte elements
  for (uint32_t b = done + 4 * lane; b < n; b += 128) {
    uint32_t acc = __ldcg(reinterpret_cast<const unsigned int *>(reinterpret_cast<const char *>(ptrs[0]) + lo + b));
    for (uint32_t q = 1; q < nsrc; ++q) {
      const uint32_t v = __ldcg(reinterpret_cast<const unsigned int *>(reinterpret_cast<const char *>(ptrs[q]) + lo + b));
      if (dt == HICCL_F32)
        acc = __float_as_uint(__fadd_rn(__uint_as_float(acc), __uint_as_float(v)));
      else
        acc += v;
    }
    *reinterpret_cast<uint32_t *>(dst + b) = acc;
  }
}

// ---------------------------------------------------------------------------
// the persistent executor
// ---------------------------------------------------------------------------

constexpr int PMAX = 8;   // pointers of a step staged in shared memory (more: read from global)

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) hiccl_exec_kernel(const DevTable T) {
  constexpr int NW = NT / 32;   // warps per CTA
  __shared__ DevEntry s_ent[MAX_ENTRIES_PER_ITEM];
  __shared__ uint32_t s_pre[MAX_ENTRIES_PER_ITEM + 1];
  __shared__ uint32_t s_meta[MAX_ENTRIES_PER_ITEM];
  __shared__ uint32_t s_poff[MAX_ENTRIES_PER_ITEM];
  __shared__ unsigned long long s_nb[MAX_ENTRIES_PER_ITEM];
  __shared__ unsigned long long s_ptr[MAX_ENTRIES_PER_ITEM][PMAX];
  __shared__ unsigned long long s_item, s_next;
  __shared__ int s_abort;
  __shared__ uint32_t s_nent;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long epoch = ld_relaxed(&T.ctl->epoch) + 1;   // this launch

  if (tid == 0) {
    s_item = atomicAdd(&T.ctl->ticket, 1ull);
    s_abort = ld_relaxed(&T.ctl->err) != 0ull;
  }
  __syncthreads();
  for (;;) {
    const unsigned long long item = s_item;
    if (item >= T.nitems || s_abort) break;

    // phase A: stage the item's entries, step descriptors and pointers in
    // shared memory and wait for the steps' predecessors (warp 0); claim the
    // next item meanwhile (warp 1), so its ticket latency is hidden
    if (warp == 0) {
      const uint32_t e0 = ldg_ro(T.item_off + item), e1 = ldg_ro(T.item_off + item + 1);
      const uint32_t ne = e1 - e0;
      uint32_t cnt = 0, s = 0;
      if (lane < (int)ne) {
        const DevEntry e = T.entries[e0 + lane];
        s = e.step;
        const uint32_t meta = ldg_ro(T.meta + s), po = ldg_ro(T.ptr_off + s);
        s_ent[lane] = e;
        s_meta[lane] = meta;
        s_poff[lane] = po;
        s_nb[lane] = ldg_ro(T.nbytes + s);
        const uint32_t np = meta_nsrc(meta) + meta_ndst(meta);
        if (np <= PMAX)
          for (uint32_t q = 0; q < np; ++q) s_ptr[lane][q] = ldg_ro(T.ptrs + po + q);
        cnt = e.seg_hi - e.seg_lo;
      }
      uint32_t inc = cnt;   // inclusive warp scan of segment counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
      }
      if (lane < (int)ne) s_pre[lane + 1] = inc;
      if (lane == 0) {
        s_pre[0] = 0;
        s_nent = ne;
      }
      if (lane < (int)ne) {
        const unsigned long long target = (unsigned long long)ldg_ro(T.indeg + s) * epoch;
        if (target && ld_acquire(T.dep + s) < target) {
          const unsigned long long t0 = global_ns();
          unsigned ns = 32;
          while (ld_acquire(T.dep + s) < target) {
            if (ld_relaxed(&T.ctl->err)) {
              s_abort = 1;
              break;
            }
            if (global_ns() - t0 > T.timeout_ns) {
              raise_error(T, ((unsigned long long)ERR_TIMEOUT << 32) | s);
              s_abort = 1;
              break;
            }
            __nanosleep(ns);
            if (ns < 256) ns <<= 1;
          }
        }
      }
    } else if (tid == 32) {
      s_next = atomicAdd(&T.ctl->ticket, 1ull);
      if (ld_relaxed(&T.ctl->err)) s_abort = 1;
    }
    __syncthreads();
    if (s_abort) break;

    // phase B: move the data; warp w takes segments w, w + NW, ... of the item
    const uint32_t total = s_pre[s_nent];
    uint32_t k = 0;
    for (uint32_t j = warp; j < total; j += NW) {
      while (s_pre[k + 1] <= j) ++k;
      const unsigned long long seg = s_ent[k].seg_lo + (j - s_pre[k]);
      const unsigned long long lo = seg * SEG_BYTES;
      const uint32_t n = (uint32_t)min((unsigned long long)SEG_BYTES, s_nb[k] - lo);
      const uint32_t meta = s_meta[k];
      const uint32_t np = meta_nsrc(meta) + meta_ndst(meta);
      const unsigned long long *ptrs = np <= PMAX ? s_ptr[k] : T.ptrs + s_poff[k];
      if (meta_op(meta) == OP_COPY)
        warp_copy(ptrs, meta_ndst(meta), lo, n, meta_aligned(meta), lane);
      else
        warp_reduce(ptrs, meta_nsrc(meta), meta_dtype(meta), lo, n, meta_aligned(meta), lane);
    }
    __syncthreads();

    // phase C: the last entry of a step releases its successors
    if (tid < (int)s_nent) {
      const uint32_t s = s_ent[tid].step;
      __threadfence();
      const unsigned long long old = atom_acq_rel_add(T.done + s, 1ull);
      if (old + 1 == (unsigned long long)ldg_ro(T.nent + s) * epoch) {
        __threadfence();
        const uint32_t a = ldg_ro(T.succ_off + s), b = ldg_ro(T.succ_off + s + 1);
        for (uint32_t q = a; q < b; ++q) red_release_add(T.dep + ldg_ro(T.succ + q), 1ull);
      }
    }
    if (tid == 0) s_item = s_next;
    __syncthreads();
  }

  // the last CTA out re-arms the control block for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned long long prev = atomicAdd(&T.ctl->exited, 1ull);
    if (prev == gridDim.x - 1) {
      T.ctl->ticket = 0;
      T.ctl->exited = 0;
      __threadfence();
      if (ld_relaxed(&T.ctl->err) == 0ull) T.ctl->epoch = epoch;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static hiccl_status_t cuda_fail(hiccl_comm *c, cudaError_t e, const char *what) {
  return fail(c, HICCL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void dev_release(hiccl_comm *c) {
  DevState *d = c->dev;
  if (!d) return;
  if (c->state == hiccl_comm::RUNNING && d->done_ev) cudaEventSynchronize(d->done_ev);
  if (d->done_ev) cudaEventDestroy(d->done_ev);
  if (d->table) cudaFree(d->table);
  if (d->counters) cudaFree(d->counters);
  if (d->scratch) cudaFree(d->scratch);
  if (d->host_err) cudaFreeHost(d->host_err);
  delete d;
  c->dev = nullptr;
}

hiccl_status_t dev_upload(hiccl_comm *c) {
  const Plan &p = c->plan;
  dev_release(c);
  DevState *d = new (std::nothrow) DevState();
  if (!d) return fail(c, HICCL_ERR_NOMEM, "host allocation");
  c->dev = d;
  cudaError_t e;
  if ((e = cudaGetDevice(&d->device)) != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&d->nsm, cudaDevAttrMultiProcessorCount, d->device)) != cudaSuccess)
    return cuda_fail(c, e, "cudaDeviceGetAttribute");
  {
    const void *ks[4] = {(const void *)hiccl_exec_kernel<64>, (const void *)hiccl_exec_kernel<128>,
                         (const void *)hiccl_exec_kernel<256>, (const void *)hiccl_exec_kernel<512>};
    for (int i = 0; i < 4; ++i) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d->occ[i], ks[i], 64 << i, 0)) != cudaSuccess)
        return cuda_fail(c, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (d->occ[i] < 1) return fail(c, HICCL_ERR_CUDA, "executor kernel cannot be resident");
    }
  }

  const size_t N = p.steps.size();
  unsigned long long scratch_base = 0;
  if (p.scratch_bytes) {
    if ((e = cudaMalloc(&d->scratch, p.scratch_bytes)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HICCL_ERR_NOMEM, "relay buffers: " + std::string(cudaGetErrorString(e)));
    }
    scratch_base = (unsigned long long)(uintptr_t)d->scratch;
  }

  // host images of the device arrays
  std::vector<unsigned long long> nbytes(N), ptrs(p.locs.size());
  std::vector<uint32_t> meta(N), ptr_off(N), indeg(N);
  for (size_t k = 0; k < p.locs.size(); ++k)
    ptrs[k] = p.locs[k].scratch ? scratch_base + p.locs[k].addr : p.locs[k].addr;
  for (size_t i = 0; i < N; ++i) {
    const HStep &st = p.steps[i];
    nbytes[i] = st.nbytes;
    ptr_off[i] = st.loc0;
    indeg[i] = p.pred_off[i + 1] - p.pred_off[i];
    bool al = true;
    for (uint32_t k = 0; k < st.nsrc + st.ndst; ++k) al = al && (ptrs[st.loc0 + k] % 16 == 0);
    // the unaligned reduce path moves 4-byte elements
    if (st.kind == OP_REDUCE && !al && c->esize != 4)
      return fail(c, HICCL_ERR_UNSUPPORTED, "reduction buffers must be 16-byte aligned for this dtype");
    meta[i] = meta_pack(st.kind, (uint32_t)c->dtype, al ? 1u : 0u, st.nsrc, st.ndst);
  }

  // one allocation for all read-only arrays
  size_t off = 0;
  auto place = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t o_nbytes = place(N * 8), o_meta = place(N * 4), o_ptroff = place(N * 4), o_indeg = place(N * 4),
               o_nent = place(N * 4), o_succoff = place((N + 1) * 4), o_succ = place(p.succ.size() * 4),
               o_ptrs = place(ptrs.size() * 8), o_ent = place(p.entries.size() * sizeof(DevEntry)),
               o_item = place(p.item_off.size() * 4);
  std::vector<char> img(std::max<size_t>(off, 256), 0);
  auto put = [&](size_t o, const void *src, size_t bytes) {
    if (bytes) std::memcpy(img.data() + o, src, bytes);
  };
  put(o_nbytes, nbytes.data(), N * 8);
  put(o_meta, meta.data(), N * 4);
  put(o_ptroff, ptr_off.data(), N * 4);
  put(o_indeg, indeg.data(), N * 4);
  put(o_nent, p.nent.data(), N * 4);
  put(o_succoff, p.succ_off.data(), (N + 1) * 4);
  put(o_succ, p.succ.data(), p.succ.size() * 4);
  put(o_ptrs, ptrs.data(), ptrs.size() * 8);
  put(o_ent, p.entries.data(), p.entries.size() * sizeof(DevEntry));
  put(o_item, p.item_off.data(), p.item_off.size() * 4);
  if ((e = cudaMalloc(&d->table, img.size())) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HICCL_ERR_NOMEM, "step table: " + std::string(cudaGetErrorString(e)));
  }
  if ((e = cudaMemcpy(d->table, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(c, e, "upload step table");

  d->counters_bytes = N * 16 + sizeof(DevCtl);
  if ((e = cudaMalloc(&d->counters, d->counters_bytes)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HICCL_ERR_NOMEM, "counters: " + std::string(cudaGetErrorString(e)));
  }
  if ((e = cudaMemset(d->counters, 0, d->counters_bytes)) != cudaSuccess) return cuda_fail(c, e, "cudaMemset");
  if ((e = cudaHostAlloc((void **)&d->host_err, sizeof(unsigned long long), cudaHostAllocMapped)) != cudaSuccess)
    return cuda_fail(c, e, "cudaHostAlloc");
  *d->host_err = 0;
  if ((e = cudaHostGetDevicePointer((void **)&d->host_err_dev, d->host_err, 0)) != cudaSuccess)
    return cuda_fail(c, e, "cudaHostGetDevicePointer");
  if ((e = cudaEventCreateWithFlags(&d->done_ev, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(c, e, "cudaEventCreate");

  char *tb = static_cast<char *>(d->table);
  char *cb = static_cast<char *>(d->counters);
  DevTable &t = d->t;
  t.nbytes = reinterpret_cast<const unsigned long long *>(tb + o_nbytes);
  t.meta = reinterpret_cast<const uint32_t *>(tb + o_meta);
  t.ptr_off = reinterpret_cast<const uint32_t *>(tb + o_ptroff);
  t.indeg = reinterpret_cast<const uint32_t *>(tb + o_indeg);
  t.nent = reinterpret_cast<const uint32_t *>(tb + o_nent);
  t.succ_off = reinterpret_cast<const uint32_t *>(tb + o_succoff);
  t.succ = reinterpret_cast<const uint32_t *>(tb + o_succ);
  t.ptrs = reinterpret_cast<const unsigned long long *>(tb + o_ptrs);
  t.entries = reinterpret_cast<const DevEntry *>(tb + o_ent);
  t.item_off = reinterpret_cast<const uint32_t *>(tb + o_item);
  t.dep = reinterpret_cast<unsigned long long *>(cb);
  t.done = reinterpret_cast<unsigned long long *>(cb + N * 8);
  t.ctl = reinterpret_cast<DevCtl *>(cb + N * 16);
  t.host_err = d->host_err_dev;
  t.nitems = p.item_off.size() - 1;
  t.timeout_ns = c->timeout_ns;
  d->indeg = std::move(indeg);
  d->indeg_dev = reinterpret_cast<uint32_t *>(tb + o_indeg);
  return HICCL_OK;
}

}  // namespace hiccl

using namespace hiccl;

extern "C" {

hiccl_status_t hiccl_start(hiccl_comm_t c, void *stream) {
  if (!c) return HICCL_ERR_INVALID;
  if (c->state == hiccl_comm::RUNNING) return fail(c, HICCL_ERR_STATE, "previous start not waited on");
  if (c->state != hiccl_comm::READY || !c->dev) return fail(c, HICCL_ERR_STATE, "start before init");
  DevState *d = c->dev;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  *d->host_err = 0;
  DevTable t = d->t;
  t.timeout_ns = c->timeout_ns;
  if (t.nitems > 0) {
    const int nt = c->threads;
    const int ti = nt == 64 ? 0 : nt == 128 ? 1 : nt == 256 ? 2 : 3;
    const int per_sm = std::min(c->ctas_per_sm, d->occ[ti]);
    const unsigned long long grid = std::min<unsigned long long>(t.nitems, (unsigned long long)d->nsm * per_sm);
    switch (nt) {
      case 64: hiccl_exec_kernel<64><<<(unsigned)grid, 64, 0, s>>>(t); break;
      case 128: hiccl_exec_kernel<128><<<(unsigned)grid, 128, 0, s>>>(t); break;
      case 256: hiccl_exec_kernel<256><<<(unsigned)grid, 256, 0, s>>>(t); break;
      default: hiccl_exec_kernel<512><<<(unsigned)grid, 512, 0, s>>>(t); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "executor launch");
  }
  cudaError_t e = cudaEventRecord(d->done_ev, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
  c->state = hiccl_comm::RUNNING;
  return HICCL_OK;
}

hiccl_status_t hiccl_wait(hiccl_comm_t c) {
  if (!c) return HICCL_ERR_INVALID;
  if (c->state != hiccl_comm::RUNNING) return fail(c, HICCL_ERR_STATE, "wait without start");
  DevState *d = c->dev;
  cudaError_t e = cudaEventSynchronize(d->done_ev);
  c->state = hiccl_comm::READY;
  if (e != cudaSuccess) return cuda_fail(c, e, "executor");
  const unsigned long long err = *(volatile unsigned long long *)d->host_err;
  if (err) {
    // the aborted launch left the counters mid-way: re-arm everything
    cudaError_t e2 = cudaMemset(d->counters, 0, d->counters_bytes);
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "counter reset");
    *d->host_err = 0;
    const unsigned code = (unsigned)(err >> 32), step = (unsigned)(err & 0xffffffffu);
    if (code == ERR_TIMEOUT)
      return fail(c, HICCL_ERR_TIMEOUT, "dependency wait of step " + std::to_string(step) + " timed out");
    return fail(c, HICCL_ERR_CUDA, "executor error " + std::to_string(code));
  }
  return HICCL_OK;
}

hiccl_status_t hiccl_debug_withhold(hiccl_comm_t c, unsigned long long index, int extra) {
  if (!c) return HICCL_ERR_INVALID;
  if (c->state != hiccl_comm::READY || !c->dev) return fail(c, HICCL_ERR_STATE, "needs an idle initialized communicator");
  DevState *d = c->dev;
  if (index >= d->indeg.size() || extra < 0 || extra > 1000) return fail(c, HICCL_ERR_INVALID, "bad step or count");
  uint32_t v = d->indeg[index] + (uint32_t)extra;
  cudaError_t e = cudaMemcpy(d->indeg_dev + index, &v, sizeof(v), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
  return HICCL_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free execution (hiccl_run_static).
//
// For callers that cannot allocate device memory themselves -- code that runs
// under a caller-owned memory pool or budget, inside an allocator callback, or
// in a process whose device allocations are made by someone else -- this path
// runs a planned communicator from one fixed device array instead of the
// buffers hiccl_init allocates.  The array is a file-scope __device__
// variable: every GPU that loads this library holds its
// HICCL_STATIC_ARENA_BYTES until the process exits.  The same persistent
// executor kernel runs on it; only where its tables live differs.
// ===========================================================================

namespace hiccl {

static __device__ __align__(256) unsigned char g_static_arena[HICCL_STATIC_ARENA_BYTES];

constexpr int MAX_STATIC_DEVICES = 64;
static void *g_static_addr[MAX_STATIC_DEVICES];   // device address of the arena, per device

// Expands the raw plan (steps, locations, predecessor offsets) copied into the
// arena into the executor's table arrays; relay offsets become arena addresses.
__global__ void hiccl_static_expand(const HStep *steps, const Loc *locs, const uint32_t *pred_off,
                                    unsigned long long nsteps, unsigned long long nlocs, uint32_t dtype,
                                    unsigned long long relay_base, unsigned long long *nbytes,
                                    uint32_t *meta, uint32_t *ptr_off, uint32_t *indeg,
                                    unsigned long long *ptrs) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (unsigned long long k = t0; k < nlocs; k += stride)
    ptrs[k] = locs[k].scratch ? relay_base + locs[k].addr : locs[k].addr;
  for (unsigned long long i = t0; i < nsteps; i += stride) {
    const HStep st = steps[i];
    bool al = true;
    for (uint32_t k = 0; k < st.nsrc + st.ndst; ++k) {
      const Loc l = locs[st.loc0 + k];
      const unsigned long long a = l.scratch ? relay_base + l.addr : l.addr;
      al = al && (a % 16 == 0);
    }
    nbytes[i] = st.nbytes;
    ptr_off[i] = st.loc0;
    indeg[i] = pred_off[i + 1] - pred_off[i];
    meta[i] = meta_pack(st.kind, dtype, al ? 1u : 0u, st.nsrc, st.ndst);
  }
}

}  // namespace hiccl

extern "C" hiccl_status_t hiccl_run_static(hiccl_comm_t c, void *stream) {
  if (!c) return HICCL_ERR_INVALID;
  if (!c->plan.valid) return HICCL_ERR_STATE;
  const Plan &p = c->plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned long long N = p.steps.size(), NL = p.locs.size(), NE = p.entries.size();
  const unsigned long long NI = p.item_off.size() ? p.item_off.size() - 1 : 0, NS = p.succ.size();
  unsigned long long off = 0;
  auto place = [&](unsigned long long bytes) {
    const unsigned long long o = off;
    off = (off + bytes + 255) & ~255ull;
    return o;
  };
  const unsigned long long o_steps = place(N * sizeof(HStep)), o_locs = place(NL * sizeof(Loc)),
                           o_predoff = place((N + 1) * 4), o_nbytes = place(N * 8), o_meta = place(N * 4),
                           o_ptroff = place(N * 4), o_indeg = place(N * 4), o_nent = place(N * 4),
                           o_succoff = place((N + 1) * 4), o_succ = place(NS * 4), o_ptrs = place(NL * 8),
                           o_ent = place(NE * sizeof(DevEntry)), o_item = place((NI + 1) * 4),
                           o_ctr = place(N * 16 + sizeof(DevCtl) + 8), o_relay = place(p.scratch_bytes);
  if (off > HICCL_STATIC_ARENA_BYTES) return HICCL_ERR_TOO_LARGE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HICCL_ERR_CUDA;
  if (dev < 0 || dev >= MAX_STATIC_DEVICES) return HICCL_ERR_UNSUPPORTED;
  if (!g_static_addr[dev]) {   // once per device, with that device current
    void *addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_static_arena) != cudaSuccess || !addr) {
      cudaGetLastError();
      return HICCL_ERR_CUDA;
    }
    g_static_addr[dev] = addr;
  }
  char *base = static_cast<char *>(g_static_addr[dev]);
  if (N == 0) return HICCL_OK;

  auto h2d = [&](unsigned long long o, const void *src, unsigned long long bytes) {
    return bytes ? cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = h2d(o_steps, p.steps.data(), N * sizeof(HStep));
  if (e == cudaSuccess) e = h2d(o_locs, p.locs.data(), NL * sizeof(Loc));
  if (e == cudaSuccess) e = h2d(o_predoff, p.pred_off.data(), (N + 1) * 4);
  if (e == cudaSuccess) e = h2d(o_nent, p.nent.data(), N * 4);
  if (e == cudaSuccess) e = h2d(o_succoff, p.succ_off.data(), (N + 1) * 4);
  if (e == cudaSuccess) e = h2d(o_succ, p.succ.data(), NS * 4);
  if (e == cudaSuccess) e = h2d(o_ent, p.entries.data(), NE * sizeof(DevEntry));
  if (e == cudaSuccess) e = h2d(o_item, p.item_off.data(), (NI + 1) * 4);
  // every call starts from zeroed counters: the arena keeps the last call's contents
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_ctr, 0, N * 16 + sizeof(DevCtl) + 8, s);
  if (e != cudaSuccess) return HICCL_ERR_CUDA;

  hiccl_static_expand<<<(unsigned)std::min<unsigned long long>((N + NL + 255) / 256, 1024), 256, 0, s>>>(
      reinterpret_cast<const HStep *>(base + o_steps), reinterpret_cast<const Loc *>(base + o_locs),
      reinterpret_cast<const uint32_t *>(base + o_predoff), N, NL, (uint32_t)c->dtype,
      (unsigned long long)(uintptr_t)(base + o_relay), reinterpret_cast<unsigned long long *>(base + o_nbytes),
      reinterpret_cast<uint32_t *>(base + o_meta), reinterpret_cast<uint32_t *>(base + o_ptroff),
      reinterpret_cast<uint32_t *>(base + o_indeg), reinterpret_cast<unsigned long long *>(base + o_ptrs));
  if (cudaGetLastError() != cudaSuccess) return HICCL_ERR_CUDA;

  DevTable t{};
  t.nbytes = reinterpret_cast<const unsigned long long *>(base + o_nbytes);
  t.meta = reinterpret_cast<const uint32_t *>(base + o_meta);
  t.ptr_off = reinterpret_cast<const uint32_t *>(base + o_ptroff);
  t.indeg = reinterpret_cast<const uint32_t *>(base + o_indeg);
  t.nent = reinterpret_cast<const uint32_t *>(base + o_nent);
  t.succ_off = reinterpret_cast<const uint32_t *>(base + o_succoff);
  t.succ = reinterpret_cast<const uint32_t *>(base + o_succ);
  t.ptrs = reinterpret_cast<const unsigned long long *>(base + o_ptrs);
  t.entries = reinterpret_cast<const DevEntry *>(base + o_ent);
  t.item_off = reinterpret_cast<const uint32_t *>(base + o_item);
  t.dep = reinterpret_cast<unsigned long long *>(base + o_ctr);
  t.done = reinterpret_cast<unsigned long long *>(base + o_ctr + N * 8);
  t.ctl = reinterpret_cast<DevCtl *>(base + o_ctr + N * 16);
  t.host_err = reinterpret_cast<unsigned long long *>(base + o_ctr + N * 16 + sizeof(DevCtl));
  t.nitems = NI;
  t.timeout_ns = c->timeout_ns;
  if (NI > 0) {
    int nsm = 0, occ = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HICCL_ERR_CUDA;
    const int nt = c->threads;
    cudaError_t oe;
    switch (nt) {
      case 64: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hiccl_exec_kernel<64>, 64, 0); break;
      case 128: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hiccl_exec_kernel<128>, 128, 0); break;
      case 256: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hiccl_exec_kernel<256>, 256, 0); break;
      default: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hiccl_exec_kernel<512>, 512, 0); break;
    }
    if (oe != cudaSuccess || occ < 1) return HICCL_ERR_CUDA;
    const unsigned grid = (unsigned)std::min<unsigned long long>(NI, (unsigned long long)nsm * std::min(c->ctas_per_sm, occ));
    switch (nt) {
      case 64: hiccl_exec_kernel<64><<<grid, 64, 0, s>>>(t); break;
      case 128: hiccl_exec_kernel<128><<<grid, 128, 0, s>>>(t); break;
      case 256: hiccl_exec_kernel<256><<<grid, 256, 0, s>>>(t); break;
      default: hiccl_exec_kernel<512><<<grid, 512, 0, s>>>(t); break;
    }
    if (cudaGetLastError() != cudaSuccess) return HICCL_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return HICCL_ERR_CUDA;
  unsigned long long err = 0;
  if (cudaMemcpy(&err, base + o_ctr + N * 16 + offsetof(DevCtl, err), sizeof(err), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return HICCL_ERR_CUDA;
  return err ? HICCL_ERR_TIMEOUT : HICCL_OK;
}
