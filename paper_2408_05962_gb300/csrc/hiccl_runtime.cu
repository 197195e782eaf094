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
// of launch e are e times the per-launch counts, and the launch index comes
// from the ticket counter itself (see DevCtl), so nothing is reset between
// starts.

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "hiccl_internal.h"

namespace hiccl {


struct DevState {
  int device = -1;
  int nsm = 0;
  int occ[4] = {0, 0, 0, 0};        // resident CTAs per SM for 128/256/512 threads (index 1..3)
  void *table = nullptr;            // read-only arrays
  void *counters = nullptr;         // dep[], done[], ctl
  size_t counters_bytes = 0;
  void *scratch = nullptr;
  unsigned long long *host_err = nullptr;
  unsigned long long *host_err_dev = nullptr;
  cudaEvent_t done_ev = nullptr;
  DevTable t{};
  std::vector<uint32_t> indeg;      // host copies, for fault injection
  std::vector<DevItem> items;
  char *recs_dev = nullptr;
  unsigned long long *trace = nullptr;   // [nitems][6] when tracing
  int err_slot = -1;
  cudaStream_t upload = nullptr;         // internal stream of the device (not owned)
  unsigned last_grid = 0;                // grid of the previous launch (its ticket arithmetic)
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
__device__ __forceinline__ void red_relaxed_add(unsigned long long *p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_relaxed_add(unsigned long long *p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
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

// one step of a fold on 32-bit lanes: f32 (IEEE RNE add, maxNum, minNum) or
// i32 (wrapping add, max, min, logical or)
__device__ __forceinline__ float comb_f(float a, float b, uint32_t rop) {
  return rop == HICCL_SUM ? __fadd_rn(a, b) : rop == HICCL_MAX ? fmaxf(a, b) : fminf(a, b);
}
__device__ __forceinline__ uint32_t comb32(uint32_t a, uint32_t b, uint32_t dt, uint32_t rop) {
  if (dt == HICCL_F32) return __float_as_uint(comb_f(__uint_as_float(a), __uint_as_float(b), rop));
  const int x = (int)a, y = (int)b;
  switch (rop) {
    case HICCL_SUM: return a + b;
    case HICCL_MAX: return (uint32_t)(x > y ? x : y);
    case HICCL_MIN: return (uint32_t)(x < y ? x : y);
    default: return (x != 0 || y != 0) ? 1u : 0u;
  }
}
__device__ __forceinline__ uint4 add4(uint4 a, uint4 b, uint32_t dt, uint32_t rop = 0) {
  if (rop == HICCL_SUM && dt == HICCL_F32) {
    a.x = __float_as_uint(__fadd_rn(__uint_as_float(a.x), __uint_as_float(b.x)));
    a.y = __float_as_uint(__fadd_rn(__uint_as_float(a.y), __uint_as_float(b.y)));
    a.z = __float_as_uint(__fadd_rn(__uint_as_float(a.z), __uint_as_float(b.z)));
    a.w = __float_as_uint(__fadd_rn(__uint_as_float(a.w), __uint_as_float(b.w)));
  } else if (rop == HICCL_SUM) {   // int32, wrapping
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
  } else {
    a.x = comb32(a.x, b.x, dt, rop);
    a.y = comb32(a.y, b.y, dt, rop);
    a.z = comb32(a.z, b.z, dt, rop);
    a.w = comb32(a.w, b.w, dt, rop);
  }
  return a;
}

// ---- reduced-precision payloads -------------------------------------------
// BF16: the upper half of a binary32; rounding to nearest even by cvt.rn.
__device__ __forceinline__ uint32_t f32_to_bf16_rn(float x) {
  unsigned short h;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
  return h;
}
// two binary32 -> two BF16 (round to nearest even) in one word; the first
// value lands in the low half
__device__ __forceinline__ uint32_t f32x2_to_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// FP8 e4m3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits, no
// infinities, S.1111.111 = NaN): four codes (byte k of w gives component k)
// -> four binary32 values, exactly.  Every e4m3 value is a binary16 value;
// binary16 -> binary32 is a mixed-precision add of -0 (x + -0 = x for every x,
// signed zeros included), measured slightly faster here than cvt.f32.f16.
__device__ __forceinline__ float4 e4m3x4_to_f32x4(uint32_t w) {
  float4 r;
  asm("{\n\t.reg .b16 lo, hi, a, b, c, d;\n\t.reg .b32 h0, h1;\n\t"
      "mov.b32 {lo, hi}, %4;\n\t"
      "cvt.rn.f16x2.e4m3x2 h0, lo;\n\tcvt.rn.f16x2.e4m3x2 h1, hi;\n\t"
      "mov.b32 {a, b}, h0;\n\tmov.b32 {c, d}, h1;\n\t"
      "add.rn.f32.f16 %0, a, 0f80000000;\n\tadd.rn.f32.f16 %1, b, 0f80000000;\n\t"
      "add.rn.f32.f16 %2, c, 0f80000000;\n\tadd.rn.f32.f16 %3, d, 0f80000000;\n\t}"
      : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
      : "r"(w));
  return r;
}
// two binary32 -> two e4m3 codes (round to nearest even, saturating at 448);
// the first value lands in the low byte
__device__ __forceinline__ uint32_t f32x2_to_e4m3x2(float lo, float hi) {
  unsigned short d;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
  return d;
}

// fold of one 16-byte vector position over f inputs, ld(q) giving input q's
// vector: f32 / i32 natively (add4), BF16 decoded to binary32, folded in
// order and rounded once
struct CombSum {
  __device__ __forceinline__ float operator()(float a, float b) const { return __fadd_rn(a, b); }
};
struct CombAny {
  uint32_t rop;
  __device__ __forceinline__ float operator()(float a, float b) const { return comb_f(a, b, rop); }
};
template <typename LD, typename COMB>
__device__ __forceinline__ uint4 fold16_bf16(LD ld, uint32_t f, COMB comb) {
  const uint4 v = ld(0);
  float a[8];
  const uint32_t w0[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[2 * i] = __uint_as_float(w0[i] << 16);
    a[2 * i + 1] = __uint_as_float(w0[i] & 0xffff0000u);
  }
#pragma unroll 2
  for (uint32_t q = 1; q < f; ++q) {
    const uint4 u = ld(q);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[2 * i] = comb(a[2 * i], __uint_as_float(w[i] << 16));
      a[2 * i + 1] = comb(a[2 * i + 1], __uint_as_float(w[i] & 0xffff0000u));
    }
  }
  uint4 r;
  r.x = f32x2_to_bf16x2(a[0], a[1]);
  r.y = f32x2_to_bf16x2(a[2], a[3]);
  r.z = f32x2_to_bf16x2(a[4], a[5]);
  r.w = f32x2_to_bf16x2(a[6], a[7]);
  return r;
}
template <typename LD>
__device__ __forceinline__ uint4 fold16(LD ld, uint32_t f, uint32_t dt, uint32_t rop = 0) {
  if (dt != HICCL_BF16) {
    uint4 v = ld(0);
    if (rop == HICCL_SUM && dt == HICCL_F32) {
#pragma unroll 4
      for (uint32_t q = 1; q < f; ++q) v = add4(v, ld(q), HICCL_F32, HICCL_SUM);
    } else {
      for (uint32_t q = 1; q < f; ++q) v = add4(v, ld(q), dt, rop);
    }
    return v;
  }
  if (rop == HICCL_SUM) return fold16_bf16(ld, f, CombSum{});
  return fold16_bf16(ld, f, CombAny{rop});
}

// FP8 blocks (128 codes, binary32 scale at byte 128, zero bytes 132..143):
// a group of 8 lanes folds one block, lane `sub` owning codes 16*sub..16*sub+15;
// blk(q) is input q's block, out the result block.  Inputs are decoded
// (code value x scale), folded in order in binary32, and the result gets a
// fresh scale amax / 448 and codes of value x (448 / amax) (both factors 1
// when amax is 0).
// All 32 lanes must call it together (the amax exchange is warp-wide);
// `active` lanes read and write.
template <typename BLK>
__device__ __forceinline__ void fp8_fold_block(BLK blk, char *out, uint32_t f, uint32_t sub, bool active) {
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  if (active) {
    {
      const char *b = blk(0);
      const uint4 c = *reinterpret_cast<const uint4 *>(b + 16 * sub);
      const float sc = *reinterpret_cast<const float *>(b + 128);
      const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 v = e4m3x4_to_f32x4(w[j]);
        acc[4 * j + 0] = __fmul_rn(v.x, sc);
        acc[4 * j + 1] = __fmul_rn(v.y, sc);
        acc[4 * j + 2] = __fmul_rn(v.z, sc);
        acc[4 * j + 3] = __fmul_rn(v.w, sc);
      }
    }
#pragma unroll 2
    for (uint32_t q = 1; q < f; ++q) {
      const char *b = blk(q);
      const uint4 c = *reinterpret_cast<const uint4 *>(b + 16 * sub);
      const float sc = *reinterpret_cast<const float *>(b + 128);
      const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 v = e4m3x4_to_f32x4(w[j]);
        acc[4 * j + 0] = __fadd_rn(acc[4 * j + 0], __fmul_rn(v.x, sc));
        acc[4 * j + 1] = __fadd_rn(acc[4 * j + 1], __fmul_rn(v.y, sc));
        acc[4 * j + 2] = __fadd_rn(acc[4 * j + 2], __fmul_rn(v.z, sc));
        acc[4 * j + 3] = __fadd_rn(acc[4 * j + 3], __fmul_rn(v.w, sc));
      }
    }
  }
  float amax = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) amax = fmaxf(amax, fabsf(acc[i]));
  amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
  amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 2));
  amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 4));
  if (!active) return;
  const float scale = amax > 0.f ? __fdiv_rn(amax, 448.f) : 1.f;
  const float inv = amax > 0.f ? __fdiv_rn(448.f, amax) : 1.f;
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t lo = f32x2_to_e4m3x2(__fmul_rn(acc[4 * i], inv), __fmul_rn(acc[4 * i + 1], inv));
    const uint32_t hi = f32x2_to_e4m3x2(__fmul_rn(acc[4 * i + 2], inv), __fmul_rn(acc[4 * i + 3], inv));
    w[i] = lo | (hi << 16);
  }
  *reinterpret_cast<uint4 *>(out + 16 * sub) = make_uint4(w[0], w[1], w[2], w[3]);
  if (sub == 0) {
    *reinterpret_cast<uint4 *>(out + 128) = make_uint4(__float_as_uint(scale), 0u, 0u, 0u);
  }
}

// copy bytes [lo, lo + n) of the source to every destination (n <= SEG_BYTES)
__device__ __forceinline__ void warp_copy(const unsigned long long *ptrs, uint32_t ndst, unsigned long long lo,
                                          uint32_t n, bool aligned, int lane) {
  const char *src = reinterpret_cast<const char *>(ptrs[0]) + lo;
  uint32_t done = 0;
  if (aligned) {
    constexpr int U = 4;   // 2 KiB per pass
    const uint32_t nvec = n >> 4;
    for (uint32_t base = 0; base < nvec; base += 32 * U) {
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = base + u * 32 + lane;
        if (i < nvec) v[u] = ld16(src + (i << 4));
      }
      for (uint32_t k = 0; k < ndst; ++k) {
        char *dst = reinterpret_cast<char *>(ptrs[1 + k]) + lo;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t i = base + u * 32 + lane;
          if (i < nvec) st16(dst + (i << 4), v[u]);
        }
      }
    }
    done = nvec << 4;
  }
  if (!aligned) {   // 4-byte words when every operand allows them
    bool w4 = (reinterpret_cast<uintptr_t>(src) & 3u) == 0;
    for (uint32_t k = 0; k < ndst; ++k) w4 = w4 && ((ptrs[1 + k] + lo) & 3u) == 0;
    if (w4) {
      const uint32_t nw = n >> 2;
      for (uint32_t i = lane; i < nw; i += 32) {
        const unsigned int v = __ldcg(reinterpret_cast<const unsigned int *>(src) + i);
        for (uint32_t k = 0; k < ndst; ++k) reinterpret_cast<unsigned int *>(reinterpret_cast<char *>(ptrs[1 + k]) + lo)[i] = v;
      }
      done = nw << 2;
    }
  }
  for (uint32_t b = done + lane; b < n; b += 32) {
    const char v = __ldcg(src + b);
    for (uint32_t k = 0; k < ndst; ++k) (reinterpret_cast<char *>(ptrs[1 + k]) + lo)[b] = v;
  }
}

// out[lo, lo + n) = in_0 + in_1 + ... (left fold, fixed order; n <= SEG_BYTES)
__device__ __forceinline__ void warp_reduce(const unsigned long long *ptrs, uint32_t nsrc, uint32_t dt,
                                            unsigned long long lo, uint32_t n, bool aligned, int lane,
                                            uint32_t rop = 0) {
  char *dst = reinterpret_cast<char *>(ptrs[nsrc]) + lo;
  if (dt == HICCL_FP8E4M3) {   // whole 144-byte blocks, four per warp pass
    const uint32_t nblk = n / FP8_BLOCK_BYTES, grp = lane >> 3, sub = lane & 7;
    for (uint32_t b0 = 0; b0 < nblk; b0 += 4) {
      const uint32_t blk = b0 + grp;
      const bool act = blk < nblk;
      const unsigned long long off = lo + (unsigned long long)blk * FP8_BLOCK_BYTES;
      fp8_fold_block([&](uint32_t q) { return reinterpret_cast<const char *>(ptrs[q]) + off; },
                     reinterpret_cast<char *>(ptrs[nsrc]) + off, nsrc, sub, act);
    }
    return;
  }
  uint32_t done = 0;
  if (aligned && dt != HICCL_BF16) {
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
        for (int u = 0; u < U; ++u) acc[u] = add4(acc[u], v[u], dt, rop);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = base + u * 32 + lane;
        if (i < nvec) st16(dst + (i << 4), acc[u]);
      }
    }
    done = nvec << 4;
  } else if (aligned) {   // BF16 vectors of 8 values
    const uint32_t nvec = n >> 4;
    for (uint32_t i = lane; i < nvec; i += 32)
      st16(dst + (i << 4),
           fold16([&](uint32_t q) { return ld16(reinterpret_cast<const char *>(ptrs[q]) + lo + (i << 4)); }, nsrc, dt,
                  rop));
    done = nvec << 4;
  }
  // element tail (or the whole unaligned range)
  if (dt == HICCL_BF16) {
    for (uint32_t b = done + 2 * lane; b < n; b += 64) {
      float acc = __uint_as_float((uint32_t)__ldcg(reinterpret_cast<const unsigned short *>(
                                      reinterpret_cast<const char *>(ptrs[0]) + lo + b)) << 16);
      for (uint32_t q = 1; q < nsrc; ++q)
        acc = comb_f(acc, __uint_as_float((uint32_t)__ldcg(reinterpret_cast<const unsigned short *>(
                                              reinterpret_cast<const char *>(ptrs[q]) + lo + b)) << 16),
                     rop);
      *reinterpret_cast<unsigned short *>(dst + b) = (unsigned short)f32_to_bf16_rn(acc);
    }
    return;
  }
  for (uint32_t b = done + 4 * lane; b < n; b += 128) {
    uint32_t acc = __ldcg(reinterpret_cast<const unsigned int *>(reinterpret_cast<const char *>(ptrs[0]) + lo + b));
    for (uint32_t q = 1; q < nsrc; ++q) {
      const uint32_t v = __ldcg(reinterpret_cast<const unsigned int *>(reinterpret_cast<const char *>(ptrs[q]) + lo + b));
      acc = comb32(acc, v, dt, rop);
    }
    *reinterpret_cast<uint32_t *>(dst + b) = acc;
  }
}

// Build-time settings: HICCL_NBUF work items staged ahead of the data warps
// per CTA (3 keeps two 256-thread CTAs per SM within shared memory);
// HICCL_PDL 1 lets executor launches use programmatic dependent launch.
#ifndef HICCL_NBUF
#define HICCL_NBUF 3
#endif
#ifndef HICCL_PDL
#define HICCL_PDL 1
#endif
constexpr int NBUF = HICCL_NBUF;   // work items staged ahead of the data warps

// A staged work item: the sections of its record at fixed offsets (each
// filled by one bulk copy), then the control fields.
struct __align__(16) ItemBuf {
  RecEnt ent[MAX_ENTRIES_PER_ITEM];
  uint32_t rpre[MAX_ENTRIES_PER_ITEM + 4];  // prefix sums of the runs' segment counts
  DevRun run[MAX_ENTRIES_PER_ITEM];         // data ranges (runs of contiguous entries)
  unsigned long long ptr[PTR_CAP];          // inline operand pointers
  uint32_t cmp[(2 * MAX_ENTRIES_PER_ITEM + 1 + SUCC_CAP + 3) / 4 * 4];   // completion section
  uint32_t nent;
  uint32_t nrun;
  uint32_t end;                             // no more items: leave the loop
  uint32_t nsucc;                           // inline successors, or SUCC_GLOBAL
  unsigned long long item;                  // ticket of the staged item
  unsigned long long pad;
};
static_assert(offsetof(ItemBuf, rpre) % 16 == 0 && offsetof(ItemBuf, run) % 16 == 0 &&
                  offsetof(ItemBuf, ptr) % 16 == 0 && offsetof(ItemBuf, cmp) % 16 == 0 && sizeof(ItemBuf) % 16 == 0,
              "bulk-copy destinations must be 16-byte aligned");

// operand pointers of entry k of a staged item
__device__ __forceinline__ const unsigned long long *ent_ptrs(const ItemBuf &X, uint32_t k, const DevTable &T) {
  const uint32_t po = X.ent[k].poff;
  return (po & PTR_GLOBAL) ? T.ptrs + (po & ~PTR_GLOBAL) : X.ptr + po;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of `parity` to complete; false after `limit_ns`
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// bulk asynchronous copies (TMA engine, no tensor map): global -> shared
// completing on an mbarrier, shared -> global tracked by bulk groups
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *sdst, const void *gsrc, uint32_t bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(sdst)),
               "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *gdst, const void *ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one arrival on the dependency counter of every successor succ[a..z): the
// successor indices are loaded four at a time before their updates are issued
__device__ __forceinline__ void release_succ(const DevTable &T, uint32_t a, uint32_t z) {
  for (uint32_t q = a; q < z; q += 4) {
    uint32_t t[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) t[u] = q + u < z ? ldg_ro(T.succ + q + u) : 0xffffffffu;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (t[u] != 0xffffffffu) red_relaxed_add(T.dep + t[u], 1ull);
  }
}

template <int NT>
struct ExecShape {
  static constexpr int D = NT / 32 - 2;                 // data warps
  static constexpr int NS = NT >= 512 ? 2 : 4;   // staging slots per data warp
  static constexpr int SMEM = D * NS * SEG_BYTES;       // dynamic shared memory (bytes)
};

// Locate the i-th of this warp's segments in a staged item: entry index k,
// byte offset lo in the step, bytes n and the step's pointer list.
struct SegRef {
  uint32_t k;
  unsigned long long lo;
  uint32_t n;
};
template <typename Buf>
__device__ __forceinline__ SegRef seg_of(const Buf &B, uint32_t j, unsigned long long segb) {
  uint32_t k = 0, hi = B.nrun;   // largest k with rpre[k] <= j
  while (hi - k > 1) {
    const uint32_t mid = (k + hi) >> 1;
    if (B.rpre[mid] <= j) k = mid;
    else hi = mid;
  }
  SegRef r;
  const DevRun &run = B.run[k];
  r.k = run.entry;
  const unsigned long long s = j - B.rpre[k];
  r.lo = run.off + s * segb;
  r.n = (uint32_t)min(segb, run.bytes - s * segb);
  return r;
}

// Warp-specialized persistent executor.  Warp 0 (control) claims work items
// in ticket order, stages each into one of NBUF shared-memory buffers and
// waits for the steps' predecessors; warps 2.. (data) move the staged item's
// segments; warp 1 (completion) waits until the data warps are done with an
// item, then releases the successors of the steps it finished and frees the
// buffer.  The three roles are chained by mbarriers (full -> done -> empty),
// so staging and dependency signalling overlap the data movement.  Only the
// control warp waits on other items, and nothing it waits for depends on it.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) hiccl_exec_kernel(const DevTable T) {
  constexpr int D = ExecShape<NT>::D;     // data warps
  constexpr int NS = ExecShape<NT>::NS;   // staging slots per data warp
  static_assert(D >= 1, "need at least one data warp");
  __shared__ ItemBuf buf[NBUF];
  __shared__ __align__(8) unsigned long long full_bar[NBUF], done_bar[NBUF], empty_bar[NBUF], rec_bar[NBUF];
  __shared__ __align__(8) unsigned long long ld_bar[D][NS];
  __shared__ __align__(8) unsigned long long red_bar[D];
  __shared__ unsigned long long s_epoch;
  extern __shared__ __align__(128) unsigned char stage[];   // D x NS x SEG_BYTES

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long limit = 2 * T.timeout_ns + 1000000ull;    // bound of the in-CTA waits
  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&full_bar[b], 32);
      mbar_init(&done_bar[b], D * 32);
      mbar_init(&empty_bar[b], 32);
      mbar_init(&rec_bar[b], 1);
    }
    for (int w = 0; w < D; ++w) {
      for (int k = 0; k < NS; ++k) mbar_init(&ld_bar[w][k], 1);
      mbar_init(&red_bar[w], 1);
    }
  }
  __syncthreads();
  // tickets of this launch: [launch0, launch0 + per_launch), the first nitems
  // of them naming work items (see DevCtl)
  const unsigned long long per_launch = T.nitems + gridDim.x;
  unsigned long long epoch = 0;   // this launch, counted from 1 (dependency targets scale with it)
  // Everything but the control warp waits here until the previous kernel of
  // the stream has completed and its writes are visible.  The control warp
  // first claims its first item and stages its record (read-only table data
  // and the ticket counter, which no other kernel uses while this one may
  // start), overlapping the previous kernel's tail, and waits before it reads
  // a dependency counter or hands the item to the data warps.
  if (warp != 0) asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == 0) {
    // ---- control: claim, stage, wait for predecessors ----
    // The ticket of the next item is claimed, and its record descriptor read
    // and its record prefetched into L2, while the current item's record is
    // in flight and its predecessors are awaited.
    unsigned long long nxt = 0;
    DevItem nd{0, 0, 0, 0, 0, {0, 0, 0}};
    if (lane == 0) nxt = atomicAdd(&T.ctl->ticket, 1ull);
    nxt = __shfl_sync(0xffffffffu, nxt, 0);
    const unsigned long long launch0 = nxt / per_launch * per_launch;
    epoch = nxt / per_launch + 1;
    if (lane == 0) s_epoch = epoch;   // read by the completion warp after the first hand-over
    nxt -= launch0;
    if (nxt < T.nitems) nd = T.items[nxt];
    for (uint32_t r = 0;; ++r) {
      const int b = r % NBUF;
      const uint32_t ph = (r / NBUF) & 1u;
      ItemBuf &B = buf[b];
      bool stop = false;
      if (r >= NBUF && !mbar_wait(&empty_bar[b], ph ^ 1u, limit)) {
        if (lane == 0) raise_error(T, (unsigned long long)ERR_STALL << 32);
        stop = true;
      }
      const unsigned long long t_claim = T.trace ? global_ns() : 0ull;
      const unsigned long long item = nxt;
      const DevItem it = nd;
      if (!stop && item >= T.nitems) {
        stop = true;
        // no more items for this CTA: the next kernel of the stream may start
        // its launch (it waits for this grid's completion before any access)
        if (lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
      }
      if (!stop) stop = ld_relaxed(&T.ctl->err) != 0ull;
      if (!stop) {
        if (lane == 0) {
          const unsigned char *src = T.recs + (size_t)it.rec * 16;
          const uint32_t be = rec_ent_bytes(it.nent), br = rec_rpre_bytes(it.nrun), bu = rec_run_bytes(it.nrun),
                         bp = rec_ptr_bytes(it.nptr), bc = rec_cmp_bytes(it.nent, it.nsucc);
          mbar_expect_tx(&rec_bar[b], be + br + bu + bp + bc);
          bulk_g2s(B.ent, src, be, &rec_bar[b]);
          bulk_g2s(B.rpre, src + be, br, &rec_bar[b]);
          if (bu) bulk_g2s(B.run, src + be + br, bu, &rec_bar[b]);
          if (bp) bulk_g2s(B.ptr, src + be + br + bu, bp, &rec_bar[b]);
          bulk_g2s(B.cmp, src + be + br + bu + bp, bc, &rec_bar[b]);
          B.nent = it.nent;
          B.nrun = it.nrun;
          B.nsucc = it.nsucc;
          nxt = atomicAdd(&T.ctl->ticket, 1ull);
        }
        nxt = __shfl_sync(0xffffffffu, nxt, 0) - launch0;
        if (nxt < T.nitems) {
          nd = T.items[nxt];
          const unsigned char *q = T.recs + (size_t)nd.rec * 16;
          const uint32_t nb = rec_bytes(nd);
          for (uint32_t o = (uint32_t)lane * 128u; o < nb; o += 32u * 128u) prefetch_l2(q + o);
        }
        if (!mbar_wait(&rec_bar[b], ph, limit)) {
          if (lane == 0) raise_error(T, (unsigned long long)ERR_STALL << 32);
          stop = true;
        }
      }
      if (r == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
      if (!stop) {
        bool bad = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t x = lane + 32 * h;
          if (x < it.nent && !bad) {
            const RecEnt e = B.ent[x];
            const unsigned long long target = (unsigned long long)e.indeg * epoch;
            if (target && ld_acquire(T.dep + e.step) < target) {
              const unsigned long long t0 = global_ns();
              unsigned ns = 32;
              while (ld_acquire(T.dep + e.step) < target) {
                if (ld_relaxed(&T.ctl->err)) {
                  bad = true;
                  break;
                }
                if (global_ns() - t0 > T.timeout_ns) {
                  raise_error(T, ((unsigned long long)ERR_TIMEOUT << 32) | e.step);
                  bad = true;
                  break;
                }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
              }
            }
          }
        }
        stop = __any_sync(0xffffffffu, bad);
      }
      if (lane == 0) {
        B.end = stop ? 1u : 0u;
        if (!stop) B.item = item;
        if (T.trace && !stop) {
          T.trace[item * 6 + 0] = t_claim;
          T.trace[item * 6 + 1] = global_ns();
          unsigned smid;
          asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
          T.trace[item * 6 + 4] = smid;
          T.trace[item * 6 + 5] = B.ent[0].step;
        }
      }
      __syncwarp();
      mbar_arrive(&full_bar[b]);
      if (stop) break;
    }
  } else if (warp == 1) {
    // ---- completion: release the successors of finished steps ----
    for (uint32_t r = 0;; ++r) {
      const int b = r % NBUF;
      const uint32_t ph = (r / NBUF) & 1u;
      ItemBuf &B = buf[b];
      if (!mbar_wait(&full_bar[b], ph, limit)) {
        if (lane == 0) raise_error(T, (unsigned long long)ERR_STALL << 32);
        break;
      }
      if (B.end) break;
      if (r == 0) epoch = s_epoch;   // written by the control warp before its first hand-over
      if (!mbar_wait(&rec_bar[b], ph, limit) || !mbar_wait(&done_bar[b], ph, limit)) {
        if (lane == 0) raise_error(T, (unsigned long long)ERR_STALL << 32);
        break;
      }
      if (T.trace && lane == 0) T.trace[B.item * 6 + 2] = global_ns();
      // fence-based release: one fence orders this item's data before the
      // counter updates; the last finisher of a step fences again (acquiring
      // the other finishers' data) before it releases the step's successors
      // Both halves of the item's (at most 64) entries are handled at once:
      // the counter updates and the loads they need are all in flight together.
      static_assert(MAX_ENTRIES_PER_ITEM <= 64, "two entries per lane");
      __threadfence();
      {
        // completion targets and successor lists come from the staged record
        // (successor lists of an item with too many stay in the global table)
        const uint32_t n = B.nent;
        const bool inl = B.nsucc != SUCC_GLOBAL;
        const uint32_t *soff = B.cmp + n, *sl = B.cmp + 2 * n + 1;
        const bool v0 = (uint32_t)lane < n, v1 = (uint32_t)lane + 32 < n;
        const uint32_t s0 = v0 ? B.ent[lane].step : 0u, s1 = v1 ? B.ent[lane + 32].step : 0u;
        uint32_t t0 = 0, t1 = 0, a0 = 0, z0 = 0, a1 = 0, z1 = 0;
        unsigned long long o0 = 0, o1 = 0;
        // a step covered by this entry alone needs no counter: this item
        // finishes it, and the fence above already orders its data before
        // the successors' updates below
        if (v0) {
          t0 = B.cmp[lane];
          a0 = inl ? soff[lane] : ldg_ro(T.succ_off + s0);
          z0 = inl ? soff[lane + 1] : ldg_ro(T.succ_off + s0 + 1);
          if (t0 > 1) o0 = atom_relaxed_add(T.done + s0, 1ull);
        }
        if (v1) {
          t1 = B.cmp[lane + 32];
          a1 = inl ? soff[lane + 32] : ldg_ro(T.succ_off + s1);
          z1 = inl ? soff[lane + 33] : ldg_ro(T.succ_off + s1 + 1);
          if (t1 > 1) o1 = atom_relaxed_add(T.done + s1, 1ull);
        }
        const bool f0 = v0 && (t0 == 1 || o0 + 1 == (unsigned long long)t0 * epoch);
        const bool f1 = v1 && (t1 == 1 || o1 + 1 == (unsigned long long)t1 * epoch);
        // the last finisher of a step split over several items acquires the
        // other finishers' data before it releases the step's successors
        if (__any_sync(0xffffffffu, (f0 && t0 > 1) || (f1 && t1 > 1))) __threadfence();
        if (inl) {
          if (f0)
            for (uint32_t q = a0; q < z0; ++q) red_relaxed_add(T.dep + sl[q], 1ull);
          if (f1)
            for (uint32_t q = a1; q < z1; ++q) red_relaxed_add(T.dep + sl[q], 1ull);
        } else {
          if (f0) release_succ(T, a0, z0);
          if (f1) release_succ(T, a1, z1);
        }
      }
      __syncwarp();
      if (T.trace && lane == 0) T.trace[B.item * 6 + 3] = global_ns();
      mbar_arrive(&empty_bar[b]);
    }
  } else {
    // ---- data: warp d moves segments d, d + D, ... of each staged item ----
    // Aligned copies go through the bulk-copy engine: each segment is loaded
    // once into one of NS staging slots and stored from there to every
    // destination.  The first loads of the next staged item are issued before
    // the current item's stores are drained, so the drain overlaps them.
    const int dw = warp - 2;
    unsigned char *my_stage = stage + (size_t)dw * NS * SEG_BYTES;
    uint32_t seq = 0;        // bulk loads issued by this warp (slot = seq % NS, phase = seq / NS)
    uint32_t pre_issued = 0; // loads of the current item issued early (during the previous item)
    uint32_t rseq = 0;       // completed phases of this warp's reduce barrier
    auto is_tma = [](const ItemBuf &X) { return meta_op(X.ent[0].meta) == OP_COPY && meta_aligned(X.ent[0].meta) != 0; };
    auto is_tma_reduce = [](const ItemBuf &X) {
      const uint32_t m = X.ent[0].meta;
      return meta_op(m) == OP_REDUCE && meta_aligned(m) != 0 && meta_nsrc(m) <= TMA_MAX_FANIN;
    };
    auto mine = [&](const ItemBuf &X) {
      const uint32_t total = X.rpre[X.nrun];
      return total > (uint32_t)dw ? (total - dw + D - 1) / D : 0u;
    };
    auto issue = [&](const ItemBuf &X, uint32_t i, uint32_t at) {   // segment i of X into load number `at`
      const SegRef g = seg_of(X, dw + i * D, T.seg);
      const unsigned long long *ptrs = ent_ptrs(X, g.k, T);
      const uint32_t slot = at % NS;
      const uint32_t n16 = g.n & ~15u;
      mbar_expect_tx(&ld_bar[dw][slot], n16);
      if (n16)
        bulk_g2s(my_stage + slot * SEG_BYTES, reinterpret_cast<const char *>(ptrs[0]) + g.lo, n16, &ld_bar[dw][slot]);
    };
    for (uint32_t r = 0;; ++r) {
      const int b = r % NBUF;
      const uint32_t ph = (r / NBUF) & 1u;
      const ItemBuf &B = buf[b];
      if (!mbar_wait(&full_bar[b], ph, limit)) {
        if (lane == 0) raise_error(T, (unsigned long long)ERR_STALL << 32);
        break;
      }
      if (B.end) break;
      if (!mbar_wait(&rec_bar[b], ph, limit)) {   // the record's bulk copies are visible to this warp
        if (lane == 0) raise_error(T, (unsigned long long)ERR_STALL << 32);
        break;
      }
      if (is_tma(B)) {
        const uint32_t nm = mine(B);
        bool stalled = false;
        if (lane == 0) {
          if (nm) {
            const uint32_t pro = nm < (uint32_t)NS ? nm : (uint32_t)NS;
            if (!pre_issued) fence_proxy_async_global();   // inputs were acquired through the generic proxy
            for (uint32_t i = pre_issued; i < pro; ++i) issue(B, i, seq + i);
            for (uint32_t i = 0; i < nm; ++i) {
              const uint32_t slot = (seq + i) % NS, par = ((seq + i) / NS) & 1u;
              if (!mbar_wait(&ld_bar[dw][slot], par, limit)) {
                raise_error(T, (unsigned long long)ERR_STALL << 32);
                stalled = true;
                break;
              }
              const SegRef g = seg_of(B, dw + i * D, T.seg);
              const uint32_t meta = B.ent[g.k].meta;
              const unsigned long long *ptrs = ent_ptrs(B, g.k, T);
              const uint32_t n16 = g.n & ~15u;
              if (n16) {
                for (uint32_t q = 0; q < meta_ndst(meta); ++q)
                  bulk_s2g(reinterpret_cast<char *>(ptrs[1 + q]) + g.lo, my_stage + slot * SEG_BYTES, n16);
                bulk_commit();
              }
              if (i + NS < nm) {
                bulk_wait_read_all();   // the slot's stores have read it
                issue(B, i + NS, seq + i + NS);
              }
            }
            if (!stalled) seq += nm;
          }
          pre_issued = 0;
          if (!stalled) {
            // start the next staged item's loads (its slots are free once the
            // stores above have read them), then drain this item's stores
            bulk_wait_read_all();
            const int b2 = (r + 1) % NBUF;
            const ItemBuf &B2 = buf[b2];
            if (mbar_try_wait(&full_bar[b2], ((r + 1) / NBUF) & 1u) && !B2.end &&
                mbar_try_wait(&rec_bar[b2], ((r + 1) / NBUF) & 1u) && is_tma(B2)) {
              const uint32_t nm2 = mine(B2);
              const uint32_t pro2 = nm2 < (uint32_t)NS ? nm2 : (uint32_t)NS;
              fence_proxy_async_global();
              for (uint32_t i = 0; i < pro2; ++i) issue(B2, i, seq + i);
              pre_issued = pro2;
            }
          }
          bulk_wait_all();             // every store of this item is complete
          fence_proxy_async_global();  // and ordered before the completion warp's generic release
        }
        if (__shfl_sync(0xffffffffu, stalled ? 1 : 0, 0)) break;
        pre_issued = __shfl_sync(0xffffffffu, pre_issued, 0);
        // ragged tails (the last few bytes of a step that are not a 16-byte multiple)
        for (uint32_t i = 0; i < nm; ++i) {
          const SegRef g = seg_of(B, dw + i * D, T.seg);
          const uint32_t n16 = g.n & ~15u;
          if (n16 == g.n) continue;
          const uint32_t meta = B.ent[g.k].meta;
          const unsigned long long *ptrs = ent_ptrs(B, g.k, T);
          if (lane < (int)(g.n - n16)) {
            const char v = __ldcg(reinterpret_cast<const char *>(ptrs[0]) + g.lo + n16 + lane);
            for (uint32_t q = 0; q < meta_ndst(meta); ++q)
              (reinterpret_cast<char *>(ptrs[1 + q]) + g.lo + n16)[lane] = v;
          }
        }
        __syncwarp();
      } else if (is_tma_reduce(B)) {
        // aligned reduces: bulk-load the f inputs of a chunk into the warp's
        // staging area, fold them in order from shared memory, and bulk-store
        // the result from shared memory
        constexpr uint32_t AREA = NS * SEG_BYTES;
        if (lane == 0) fence_proxy_async_global();   // inputs were acquired through the generic proxy
        bool stalled = false;
        const uint32_t nm = mine(B);
        for (uint32_t i = 0; i < nm && !stalled; ++i) {
          const SegRef g = seg_of(B, dw + i * D, T.seg);
          const uint32_t meta = B.ent[g.k].meta;
          const uint32_t f = meta_nsrc(meta);
          const unsigned long long *ptrs = ent_ptrs(B, g.k, T);
          const uint32_t n16 = g.n & ~15u;
          const uint32_t dt = meta_dtype(meta);
          const uint32_t chunk = dt == HICCL_FP8E4M3 ? (AREA / f) / FP8_BLOCK_BYTES * FP8_BLOCK_BYTES
                                                     : (AREA / f) & ~15u;
          for (uint32_t off = 0; off < n16; off += chunk) {
            const uint32_t len = min(chunk, n16 - off);
            if (lane == 0) {
              bulk_wait_read_all();   // the previous chunk's store has read the area
              mbar_expect_tx(&red_bar[dw], f * len);
              for (uint32_t q = 0; q < f; ++q)
                bulk_g2s(my_stage + q * chunk, reinterpret_cast<const char *>(ptrs[q]) + g.lo + off, len,
                         &red_bar[dw]);
            }
            if (!mbar_wait(&red_bar[dw], rseq & 1u, limit)) {
              if (lane == 0) raise_error(T, (unsigned long long)ERR_STALL << 32);
              stalled = true;
              break;
            }
            ++rseq;
            if (dt == HICCL_FP8E4M3) {
              const uint32_t nblk = len / FP8_BLOCK_BYTES, grp = lane >> 3, sub = lane & 7;
              for (uint32_t b0 = 0; b0 < nblk; b0 += 4) {
                const uint32_t blk = b0 + grp;
                const uint32_t boff = blk * FP8_BLOCK_BYTES;
                fp8_fold_block([&](uint32_t q) { return reinterpret_cast<const char *>(my_stage + q * chunk + boff); },
                               reinterpret_cast<char *>(my_stage + boff), f, sub, blk < nblk);
              }
            } else {
              for (uint32_t v = lane; v < len / 16; v += 32)
                *reinterpret_cast<uint4 *>(my_stage + v * 16) = fold16(
                    [&](uint32_t q) { return *reinterpret_cast<const uint4 *>(my_stage + q * chunk + v * 16); }, f, dt,
                    meta_rop(meta));
            }
            fence_proxy_async_smem();   // the folded chunk is read by the bulk store
            __syncwarp();
            if (lane == 0) {
              bulk_s2g(reinterpret_cast<char *>(ptrs[f]) + g.lo + off, my_stage, len);
              bulk_commit();
            }
          }
          // element tail of the last segment of a step (fewer than 16 bytes)
          if (!stalled && n16 != g.n && dt == HICCL_BF16 && lane < (int)((g.n - n16) / 2)) {
            const unsigned long long b = g.lo + n16 + 2 * lane;
            float acc = __uint_as_float((uint32_t)__ldcg(reinterpret_cast<const unsigned short *>(
                                            reinterpret_cast<const char *>(ptrs[0]) + b)) << 16);
            for (uint32_t q = 1; q < f; ++q)
              acc = comb_f(acc, __uint_as_float((uint32_t)__ldcg(reinterpret_cast<const unsigned short *>(
                                                    reinterpret_cast<const char *>(ptrs[q]) + b)) << 16),
                           meta_rop(meta));
            *reinterpret_cast<unsigned short *>(reinterpret_cast<char *>(ptrs[f]) + b) = (unsigned short)f32_to_bf16_rn(acc);
          } else if (!stalled && n16 != g.n && dt != HICCL_BF16 && lane < (int)((g.n - n16) / 4)) {
            const unsigned long long b = g.lo + n16 + 4 * lane;
            uint32_t acc = __ldcg(reinterpret_cast<const unsigned int *>(reinterpret_cast<const char *>(ptrs[0]) + b));
            for (uint32_t q = 1; q < f; ++q) {
              const uint32_t v = __ldcg(reinterpret_cast<const unsigned int *>(reinterpret_cast<const char *>(ptrs[q]) + b));
              acc = comb32(acc, v, dt, meta_rop(meta));
            }
            *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(ptrs[f]) + b) = acc;
          }
        }
        if (lane == 0) {
          bulk_wait_all();             // every store of this item is complete
          fence_proxy_async_global();  // and ordered before the completion warp's generic release
        }
        if (__any_sync(0xffffffffu, stalled)) break;
        __syncwarp();
      } else {
        const uint32_t rtotal = B.rpre[B.nrun];
        for (uint32_t j = dw; j < rtotal; j += D) {
          const SegRef g = seg_of(B, j, T.seg);
          const uint32_t meta = B.ent[g.k].meta;
          const unsigned long long *ptrs = ent_ptrs(B, g.k, T);
          if (meta_op(meta) == OP_COPY)
            warp_copy(ptrs, meta_ndst(meta), g.lo, g.n, meta_aligned(meta), lane);
          else
            warp_reduce(ptrs, meta_nsrc(meta), meta_dtype(meta), g.lo, g.n, meta_aligned(meta), lane, meta_rop(meta));
        }
      }
      mbar_arrive(&done_bar[b]);
    }
  }

}

// ---------------------------------------------------------------------------
// launch helpers (shared by hiccl_start and hiccl_run_static)
// ---------------------------------------------------------------------------

template <int NT>
static cudaError_t exec_prepare(int *occ) {
  cudaError_t e = cudaFuncSetAttribute(hiccl_exec_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ExecShape<NT>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, hiccl_exec_kernel<NT>, NT, ExecShape<NT>::SMEM);
}

// set the kernel's shared-memory limit and return its resident CTAs per SM
static cudaError_t exec_occupancy(int nt, int *occ) {
  switch (nt) {
    case 128: return exec_prepare<128>(occ);
    case 256: return exec_prepare<256>(occ);
    default: return exec_prepare<512>(occ);
  }
}

// Launches allow programmatic dependent launch: the CTAs of this executor
// may become resident while the previous kernel of the stream drains, and
// wait (griddepcontrol.wait) for its completion before touching memory.
template <int NT>
static void exec_launch_t(unsigned grid, cudaStream_t s, const DevTable &t) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = ExecShape<NT>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = HICCL_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, hiccl_exec_kernel<NT>, t);
}
static void exec_launch(int nt, unsigned grid, cudaStream_t s, const DevTable &t) {
  switch (nt) {
    case 128: exec_launch_t<128>(grid, s, t); break;
    case 256: exec_launch_t<256>(grid, s, t); break;
    default: exec_launch_t<512>(grid, s, t); break;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// ---- process-wide resources, per device -------------------------------------
// Uploads run on an internal non-blocking stream with stream-ordered
// allocation, so creating or destroying a communicator never synchronizes the
// device with kernels other streams are running.  The mapped host error words
// come from one pinned slab.
constexpr int MAXDEV = 64;
struct DeviceRes {
  std::once_flag once;
  cudaError_t status = cudaSuccess;
  cudaStream_t upload = nullptr;
  int nsm = 0;
  int occ[4] = {0, 0, 0, 0};
};
static DeviceRes g_dev[MAXDEV];

static cudaError_t device_res(int dev, DeviceRes **out) {
  if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
  DeviceRes &r = g_dev[dev];
  std::call_once(r.once, [&]() {
    cudaError_t e = cudaStreamCreateWithFlags(&r.upload, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&r.nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 1; i < 4 && e == cudaSuccess; ++i) e = exec_occupancy(64 << i, &r.occ[i]);
    r.status = e;
  });
  *out = &r;
  return r.status;
}

static int threads_index(int nt) { return nt == 128 ? 1 : nt == 256 ? 2 : 3; }

unsigned long long exec_grid(const hiccl_comm &c) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  DeviceRes *res = nullptr;
  if (device_res(dev, &res) != cudaSuccess) return 0;
  const int occ = res->occ[threads_index(c.threads)];
  if (res->nsm < 1 || occ < 1) return 0;
  return (unsigned long long)res->nsm * (unsigned long long)std::min(c.ctas_per_sm, occ);
}

constexpr int ERR_SLOTS = 1 << 16;
static std::mutex g_err_mu;
static unsigned long long *g_err_host = nullptr, *g_err_dev = nullptr;
static std::vector<int> g_err_free;

static cudaError_t err_slot(unsigned long long **host, unsigned long long **dev, int *slot) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_host) {
    cudaError_t e = cudaHostAlloc((void **)&g_err_host, ERR_SLOTS * sizeof(unsigned long long), cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    if ((e = cudaHostGetDevicePointer((void **)&g_err_dev, g_err_host, 0)) != cudaSuccess) return e;
    g_err_free.reserve(ERR_SLOTS);
    for (int k = ERR_SLOTS - 1; k >= 0; --k) g_err_free.push_back(k);
  }
  if (g_err_free.empty()) return cudaErrorMemoryAllocation;
  *slot = g_err_free.back();
  g_err_free.pop_back();
  *host = g_err_host + *slot;
  *dev = g_err_dev + *slot;
  **host = 0;
  return cudaSuccess;
}

static void err_release(int slot) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (slot >= 0) g_err_free.push_back(slot);
}

static hiccl_status_t cuda_fail(hiccl_comm *c, cudaError_t e, const char *what) {
  return fail(c, HICCL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void dev_release(hiccl_comm *c) {
  DevState *d = c->dev;
  if (!d) return;
  if (c->state == hiccl_comm::RUNNING && d->done_ev) cudaEventSynchronize(d->done_ev);
  if (d->done_ev) cudaEventDestroy(d->done_ev);
  if (d->upload) {   // stream-ordered frees: no device-wide synchronization
    if (d->table) cudaFreeAsync(d->table, d->upload);
    if (d->counters) cudaFreeAsync(d->counters, d->upload);
    if (d->scratch) cudaFreeAsync(d->scratch, d->upload);
    if (d->trace) cudaFreeAsync(d->trace, d->upload);
  }
  err_release(d->err_slot);
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
  DeviceRes *res = nullptr;
  if ((e = device_res(d->device, &res)) != cudaSuccess) return cuda_fail(c, e, "device set-up");
  d->nsm = res->nsm;
  for (int i = 1; i < 4; ++i) {
    d->occ[i] = res->occ[i];
    if (d->occ[i] < 1) return fail(c, HICCL_ERR_CUDA, "executor kernel cannot be resident");
  }
  d->upload = res->upload;
  cudaStream_t us = d->upload;
  auto dalloc = [&](void **ptr, size_t bytes, const char *what) -> hiccl_status_t {
    cudaError_t ee = cudaMallocAsync(ptr, bytes, us);
    if (ee != cudaSuccess) {
      cudaGetLastError();
      *ptr = nullptr;
      return fail(c, HICCL_ERR_NOMEM, std::string(what) + ": " + cudaGetErrorString(ee));
    }
    return HICCL_OK;
  };

  const size_t N = p.steps.size();
  unsigned long long scratch_base = 0;
  if (p.scratch_bytes) {
    hiccl_status_t st = dalloc(&d->scratch, p.scratch_bytes, "relay buffers");
    if (st != HICCL_OK) return st;
    scratch_base = (unsigned long long)(uintptr_t)d->scratch;
  }

  // host image of the read-only arrays, in one allocation
  TableImage im;
  build_image(p, scratch_base, im);
  size_t off = 0;
  auto place = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t o_recs = place(im.recs.size()), o_items = place(im.items.size() * sizeof(DevItem)),
               o_nent = place(N * 4), o_succoff = place((N + 1) * 4), o_succ = place(p.succ.size() * 4),
               o_ptrs = place(im.ptrs.size() * 8);
  std::vector<char> img(std::max<size_t>(off, 256), 0);
  auto put = [&](size_t o, const void *src, size_t bytes) {
    if (bytes) std::memcpy(img.data() + o, src, bytes);
  };
  put(o_recs, im.recs.data(), im.recs.size());
  put(o_items, im.items.data(), im.items.size() * sizeof(DevItem));
  put(o_nent, p.nent.data(), N * 4);
  put(o_succoff, p.succ_off.data(), (N + 1) * 4);
  put(o_succ, p.succ.data(), p.succ.size() * 4);
  put(o_ptrs, im.ptrs.data(), im.ptrs.size() * 8);
  {
    hiccl_status_t st = dalloc(&d->table, img.size(), "step table");
    if (st != HICCL_OK) return st;
  }
  if ((e = cudaMemcpyAsync(d->table, img.data(), img.size(), cudaMemcpyHostToDevice, us)) != cudaSuccess)
    return cuda_fail(c, e, "upload step table");

  d->counters_bytes = N * 16 + sizeof(DevCtl);
  {
    hiccl_status_t st = dalloc(&d->counters, d->counters_bytes, "counters");
    if (st != HICCL_OK) return st;
  }
  if ((e = cudaMemsetAsync(d->counters, 0, d->counters_bytes, us)) != cudaSuccess)
    return cuda_fail(c, e, "cudaMemsetAsync");
  if ((e = err_slot(&d->host_err, &d->host_err_dev, &d->err_slot)) != cudaSuccess)
    return cuda_fail(c, e, "error word");
  if ((e = cudaEventCreateWithFlags(&d->done_ev, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(c, e, "cudaEventCreate");

  char *tb = static_cast<char *>(d->table);
  char *cb = static_cast<char *>(d->counters);
  DevTable &t = d->t;
  t.recs = reinterpret_cast<const unsigned char *>(tb + o_recs);
  t.items = reinterpret_cast<const DevItem *>(tb + o_items);
  t.nent = reinterpret_cast<const uint32_t *>(tb + o_nent);
  t.succ_off = reinterpret_cast<const uint32_t *>(tb + o_succoff);
  t.succ = reinterpret_cast<const uint32_t *>(tb + o_succ);
  t.ptrs = reinterpret_cast<const unsigned long long *>(tb + o_ptrs);
  t.dep = reinterpret_cast<unsigned long long *>(cb);
  t.done = reinterpret_cast<unsigned long long *>(cb + N * 8);
  t.ctl = reinterpret_cast<DevCtl *>(cb + N * 16);
  t.host_err = d->host_err_dev;
  t.nitems = p.item_off.size() - 1;
  t.timeout_ns = c->timeout_ns;
  t.seg = p.seg;
  t.trace = nullptr;
  if (c->trace && t.nitems) {
    hiccl_status_t st = dalloc((void **)&d->trace, t.nitems * 6 * sizeof(unsigned long long), "trace buffer");
    if (st != HICCL_OK) return st;
    t.trace = d->trace;
  }
  // the uploads must have landed before the first start (on any stream)
  if ((e = cudaStreamSynchronize(us)) != cudaSuccess) return cuda_fail(c, e, "upload");
  d->indeg = std::move(im.indeg);
  d->items = std::move(im.items);
  d->recs_dev = tb + o_recs;
  return HICCL_OK;
}

}  // namespace hiccl

using namespace hiccl;

extern "C" {

hiccl_status_t hiccl_start(hiccl_comm_t c, void *stream) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state == hiccl_comm::RUNNING) return fail(c, HICCL_ERR_STATE, "previous start not waited on");
    if (c->state != hiccl_comm::READY || !c->dev) return fail(c, HICCL_ERR_STATE, "start before init");
    DevState *d = c->dev;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaStreamIsCapturing");
    if (cap == cudaStreamCaptureStatusNone) *d->host_err = 0;
    DevTable t = d->t;
    t.timeout_ns = c->timeout_ns;
    if (t.nitems > 0) {
      const int nt = c->threads;
      const int per_sm = std::min(c->ctas_per_sm, d->occ[threads_index(nt)]);
      const unsigned long long grid = std::min<unsigned long long>(t.nitems, (unsigned long long)d->nsm * per_sm);
      // the ticket arithmetic assumes the grid of the previous launches: a
      // launch with another grid (changed options) starts from zeroed counters
      if (d->last_grid && d->last_grid != (unsigned)grid) {
        cudaError_t e = cudaMemsetAsync(d->counters, 0, d->counters_bytes, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "counter reset");
      }
      d->last_grid = (unsigned)grid;
      exec_launch(nt, (unsigned)grid, s, t);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(c, e, "executor launch");
    }
    // under stream capture only the launch is recorded: each replay of the
    // graph is a complete start (counters re-arm themselves on the device);
    // the caller synchronizes the graph launch on its stream
    if (cap != cudaStreamCaptureStatusNone) return HICCL_OK;
    cudaError_t e = cudaEventRecord(d->done_ev, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
    c->state = hiccl_comm::RUNNING;
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_wait(hiccl_comm_t c) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state != hiccl_comm::RUNNING) return fail(c, HICCL_ERR_STATE, "wait without start");
    DevState *d = c->dev;
    cudaError_t e = cudaEventSynchronize(d->done_ev);
    c->state = hiccl_comm::READY;
    if (e != cudaSuccess) return cuda_fail(c, e, "executor");
    const unsigned long long err = *(volatile unsigned long long *)d->host_err;
    if (err) {
      // the aborted launch left the counters mid-way: re-arm everything
      cudaError_t e2 = cudaMemsetAsync(d->counters, 0, d->counters_bytes, d->upload);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(d->upload);
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "counter reset");
      *d->host_err = 0;
      const unsigned code = (unsigned)(err >> 32), step = (unsigned)(err & 0xffffffffu);
      if (code == ERR_TIMEOUT)
        return fail(c, HICCL_ERR_TIMEOUT, "dependency wait of step " + std::to_string(step) + " timed out");
      if (code == ERR_STALL) return fail(c, HICCL_ERR_TIMEOUT, "an executor pipeline wait timed out");
      return fail(c, HICCL_ERR_CUDA, "executor error " + std::to_string(code));
    }
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_autotune(hiccl_comm_t c, void *stream, int flags, hiccl_tune_t *best) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->group) return fail(c, HICCL_ERR_UNSUPPORTED, "tune the members, then group them");
    if (c->state != hiccl_comm::READY || !c->dev) return fail(c, HICCL_ERR_STATE, "needs an idle initialized communicator");
    const std::vector<int> h = c->plan.hierarchy;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      return cuda_fail(c, cudaGetLastError(), "cudaEventCreate");
    }
    hiccl_tune_t cur{c->plan.stripe, c->plan.pipeline, c->order, c->threads, c->item_bytes, 0.f, 0};
    hiccl_tune_t top = cur;
    top.us = 3.4e38f;
    int trials = 0;
    // time one configuration; the communicator is left initialized with it
    auto trial = [&](const hiccl_tune_t &k, float &us) -> hiccl_status_t {
      c->order = k.order;
      c->item_bytes = k.item_bytes;
      c->threads = k.threads;
      hiccl_status_t st = replan(c, h, k.stripe, k.pipeline);
      if (st != HICCL_OK) return st;
      if ((st = dev_upload(c)) != HICCL_OK) return st;
      c->state = hiccl_comm::READY;
      float ts[4];
      for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0, s);
        if ((st = hiccl_start(c, s)) != HICCL_OK) return st;
        cudaEventRecord(e1, s);
        if ((st = hiccl_wait(c)) != HICCL_OK) return st;
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ts[r], e0, e1);
      }
      std::sort(ts + 1, ts + 4);   // run 0 is the warm-up
      us = ts[2] * 1000.f;
      ++trials;
      return HICCL_OK;
    };
    auto consider = [&](hiccl_tune_t k) -> hiccl_status_t {
      float us = 0.f;
      hiccl_status_t st = trial(k, us);
      if (st != HICCL_OK) return st;
      k.us = us;
      if (us < top.us) top = k;
      return HICCL_OK;
    };
    hiccl_status_t st = HICCL_OK;
    if (flags & 1) {   // the paper's stripe and pipeline parameters first
      std::vector<int> ss{cur.stripe, 1};
      if (!h.empty() && h.back() > 1 && h.back() <= c->P) ss.push_back(h.back());
      std::sort(ss.begin(), ss.end());
      ss.erase(std::unique(ss.begin(), ss.end()), ss.end());
      if (c->ring > 1)   // a ring keeps the stripe inside one node
        ss.erase(std::remove_if(ss.begin(), ss.end(), [&](int v) { return v > c->P / c->ring; }), ss.end());
      for (int sv : ss)
        for (int mv : {1, 2, 4, 8}) {
          hiccl_tune_t k = cur;
          k.stripe = sv;
          k.pipeline = mv;
          if (st == HICCL_OK) st = consider(k);
        }
    } else if (st == HICCL_OK) {
      st = consider(cur);
    }
    const hiccl_tune_t base = top;
    for (int order : {1, 0})
      for (unsigned long long ib : {32768ull, 49152ull, 65536ull, 131072ull}) {
        hiccl_tune_t k = base;
        k.order = order;
        k.item_bytes = ib;
        if (st == HICCL_OK && !(order == base.order && ib == base.item_bytes)) st = consider(k);
      }
    if (st == HICCL_OK) {
      float us = 0.f;
      st = trial(top, us);   // leave the communicator on the best configuration
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HICCL_OK) return st;
    top.trials = trials;
    if (best) *best = top;
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_get_trace(hiccl_comm_t c, unsigned long long *out, size_t capacity, size_t *written) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c || !written) return HICCL_ERR_INVALID;
    *written = 0;
    if (c->state != hiccl_comm::READY || !c->dev) return fail(c, HICCL_ERR_STATE, "needs an idle initialized communicator");
    DevState *d = c->dev;
    if (!d->trace) return fail(c, HICCL_ERR_STATE, "tracing is off (HICCL_OPT_TRACE)");
    const size_t n = std::min<size_t>(capacity, (size_t)d->t.nitems * 6);
    if (n && out) {
      cudaError_t e = cudaMemcpy(out, d->trace, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(c, e, "trace copy");
    }
    *written = n;
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_debug_withhold(hiccl_comm_t c, unsigned long long index, int extra) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state != hiccl_comm::READY || !c->dev) return fail(c, HICCL_ERR_STATE, "needs an idle initialized communicator");
    DevState *d = c->dev;
    if (index >= d->indeg.size() || extra < 0 || extra > 1000) return fail(c, HICCL_ERR_INVALID, "bad step or count");
    // the dependency count is stored in every record entry of the step
    uint32_t v[1] = {d->indeg[index] + (uint32_t)extra};
    const Plan &p = c->plan;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < d->items.size() && e == cudaSuccess; ++i)
      for (uint32_t k = p.item_off[i]; k < p.item_off[i + 1] && e == cudaSuccess; ++k)
        if (p.entries[k].step == index) {
          char *at = d->recs_dev + (size_t)d->items[i].rec * 16 + (size_t)(k - p.item_off[i]) * sizeof(RecEnt) +
                     offsetof(RecEnt, indeg);
          e = cudaMemcpyAsync(at, v, sizeof(uint32_t), cudaMemcpyHostToDevice, d->upload);
        }
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->upload);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync");
    return HICCL_OK;
  });
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
// device address of the arena, looked up once per device with that device
// current; a cudaDeviceReset of the device invalidates it (the lookup is not
// repeated in this process)
struct StaticAddr {
  std::once_flag once;
  cudaError_t status = cudaSuccess;
  void *addr = nullptr;
};
static StaticAddr g_static_addr[MAX_STATIC_DEVICES];

}  // namespace hiccl

extern "C" hiccl_status_t hiccl_run_static(hiccl_comm_t c, void *stream) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (!c->plan.valid) return HICCL_ERR_STATE;
    const Plan &p = c->plan;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned long long N = p.steps.size();
    const unsigned long long NI = p.item_off.size() ? p.item_off.size() - 1 : 0, NS = p.succ.size();

    // arena layout: relay buffers first (their addresses go into the records),
    // then the read-only arrays, then the counters, the control block and the
    // error word.  The sizes do not depend on where the arena lies, so a plan
    // that does not fit is rejected before any CUDA call.
    unsigned long long off = 0;
    auto place = [&](unsigned long long bytes) {
      const unsigned long long o = off;
      off = (off + bytes + 255) & ~255ull;
      return o;
    };
    const unsigned long long rec_b = record_bytes(p);
    const unsigned long long o_relay = place(p.scratch_bytes);
    const unsigned long long o_recs = place(rec_b), o_items = place(NI * sizeof(DevItem)), o_nent = place(N * 4),
                             o_succoff = place((N + 1) * 4), o_succ = place(NS * 4), o_ptrs = place(p.locs.size() * 8),
                             ctr_bytes = N * 16 + sizeof(DevCtl) + 8, o_ctr = place(ctr_bytes);
    if (off > HICCL_STATIC_ARENA_BYTES) return HICCL_ERR_TOO_LARGE;
    if (N == 0) return HICCL_OK;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HICCL_ERR_CUDA;
    if (dev < 0 || dev >= MAX_STATIC_DEVICES) return HICCL_ERR_UNSUPPORTED;
    StaticAddr &sa = g_static_addr[dev];
    std::call_once(sa.once, [&]() {   // once per device, with that device current
      void *addr = nullptr;
      sa.status = cudaGetSymbolAddress(&addr, g_static_arena);
      if (sa.status == cudaSuccess && !addr) sa.status = cudaErrorInvalidSymbol;
      if (sa.status != cudaSuccess) cudaGetLastError();
      sa.addr = addr;
    });
    if (sa.status != cudaSuccess) return HICCL_ERR_CUDA;
    char *base = static_cast<char *>(sa.addr);

    TableImage im;
    build_image(p, (unsigned long long)(uintptr_t)(base + o_relay), im);
    if (im.recs.size() != rec_b || im.items.size() != NI || im.ptrs.size() != p.locs.size()) return HICCL_ERR_INVALID;

    auto h2d = [&](unsigned long long o, const void *src, unsigned long long bytes) {
      return bytes ? cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = h2d(o_recs, im.recs.data(), im.recs.size());
    if (e == cudaSuccess) e = h2d(o_items, im.items.data(), im.items.size() * sizeof(DevItem));
    if (e == cudaSuccess) e = h2d(o_nent, p.nent.data(), N * 4);
    if (e == cudaSuccess) e = h2d(o_succoff, p.succ_off.data(), (N + 1) * 4);
    if (e == cudaSuccess) e = h2d(o_succ, p.succ.data(), NS * 4);
    if (e == cudaSuccess) e = h2d(o_ptrs, im.ptrs.data(), im.ptrs.size() * 8);
    // every call starts from zeroed counters: the arena keeps the last call's contents
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_ctr, 0, ctr_bytes, s);
    if (e != cudaSuccess) return HICCL_ERR_CUDA;

    DevTable t{};
    t.recs = reinterpret_cast<const unsigned char *>(base + o_recs);
    t.items = reinterpret_cast<const DevItem *>(base + o_items);
    t.nent = reinterpret_cast<const uint32_t *>(base + o_nent);
    t.succ_off = reinterpret_cast<const uint32_t *>(base + o_succoff);
    t.succ = reinterpret_cast<const uint32_t *>(base + o_succ);
    t.ptrs = reinterpret_cast<const unsigned long long *>(base + o_ptrs);
    t.dep = reinterpret_cast<unsigned long long *>(base + o_ctr);
    t.done = reinterpret_cast<unsigned long long *>(base + o_ctr + N * 8);
    t.ctl = reinterpret_cast<DevCtl *>(base + o_ctr + N * 16);
    t.host_err = reinterpret_cast<unsigned long long *>(base + o_ctr + N * 16 + sizeof(DevCtl));
    t.nitems = NI;
    t.timeout_ns = c->timeout_ns;
    t.seg = p.seg;
    t.trace = nullptr;
    if (NI > 0) {
      int nsm = 0, occ = 0;
      if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HICCL_ERR_CUDA;
      const int nt = c->threads;
      if (exec_occupancy(nt, &occ) != cudaSuccess || occ < 1) return HICCL_ERR_CUDA;
      const unsigned grid = (unsigned)std::min<unsigned long long>(NI, (unsigned long long)nsm * std::min(c->ctas_per_sm, occ));
      exec_launch(nt, grid, s, t);
      if (cudaGetLastError() != cudaSuccess) return HICCL_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return HICCL_ERR_CUDA;
    unsigned long long err = 0;
    if (cudaMemcpy(&err, base + o_ctr + N * 16 + offsetof(DevCtl, err), sizeof(err), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return HICCL_ERR_CUDA;
    if (!err) return HICCL_OK;
    // the same decoding as hiccl_wait: a wait that ran out is a timeout, any
    // other executor error a CUDA-side failure
    const unsigned code = (unsigned)(err >> 32);
    return (code == ERR_TIMEOUT || code == ERR_STALL) ? HICCL_ERR_TIMEOUT : HICCL_ERR_CUDA;
  });
}
