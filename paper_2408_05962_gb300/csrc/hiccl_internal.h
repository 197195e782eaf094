// Internal data structures shared by the host factorizer (hiccl_plan.cpp) and
// the device runtime (hiccl_runtime.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "../../include/hiccl.h"

#ifdef __CUDACC__
#define HICCL_HD __host__ __device__
#else
#define HICCL_HD
#endif

namespace hiccl {

// ---------------------------------------------------------------------------
// device-side layout of an uploaded plan
// ---------------------------------------------------------------------------

// A warp moves one segment of a step at a time: at most SEG_BYTES of every
// operand (the staging slot size).  FP8 steps use segments of whole 144-byte
// blocks.
constexpr uint32_t SEG_BYTES = 4096;
constexpr uint32_t FP8_BLOCK_ELEMS = 128;
constexpr uint32_t FP8_BLOCK_BYTES = 144;   // 128 e4m3 codes, binary32 scale, 12 zero bytes
HICCL_HD inline uint32_t seg_bytes_of(uint32_t dtype) { return dtype == 3u ? 28u * FP8_BLOCK_BYTES : SEG_BYTES; }
constexpr uint32_t MAX_ENTRIES_PER_ITEM = 64;
// executor CTAs assumed when a plan is made without a device to query: a
// 152-SM GB300 at two CTAs per SM
constexpr unsigned long long DEFAULT_GRID = 304;
// work-item sizing (measured on the seven collectives of 4 MiB per rank at
// P = 64): pipeline slots under SMALL_SLOT_BYTES are spread over the grid,
// larger ones over LARGE_SLOT_ITEMS items
constexpr unsigned long long SMALL_SLOT_BYTES = 12ull << 20;
constexpr unsigned long long LARGE_SLOT_ITEMS = 768;
constexpr uint32_t MAX_FANIN = 1024;    // reduce inputs / copy destinations per step
constexpr uint32_t TMA_MAX_FANIN = 8;   // reduce inputs folded in shared memory

enum : uint32_t { OP_COPY = 0, OP_REDUCE = 1 };

// meta word of a step: op (2 bits) | dtype (4) | aligned16 (1) | reduction
// operator (3) | nsrc (11) | ndst (11)
HICCL_HD inline uint32_t meta_pack(uint32_t op, uint32_t dt, uint32_t al, uint32_t nsrc, uint32_t ndst,
                                   uint32_t rop = 0) {
  return op | (dt << 2) | (al << 6) | (rop << 7) | (nsrc << 10) | (ndst << 21);
}
HICCL_HD inline uint32_t meta_op(uint32_t m) { return m & 3u; }
HICCL_HD inline uint32_t meta_dtype(uint32_t m) { return (m >> 2) & 15u; }
HICCL_HD inline uint32_t meta_aligned(uint32_t m) { return (m >> 6) & 1u; }
HICCL_HD inline uint32_t meta_rop(uint32_t m) { return (m >> 7) & 7u; }
HICCL_HD inline uint32_t meta_nsrc(uint32_t m) { return (m >> 10) & 2047u; }
HICCL_HD inline uint32_t meta_ndst(uint32_t m) { return (m >> 21) & 2047u; }

// one contiguous run of a step's segments inside a work item
struct DevEntry {
  uint32_t step;
  uint32_t seg_lo;
  uint32_t seg_hi;
  uint32_t pad;
};

// A run of an item: consecutive entries whose steps have identical shape and
// operands that continue one another in memory (adjacent pipeline channels of
// one branch), moved as one range.  `entry` is the run's first entry within
// the item; `off` the byte offset in that entry's step where the run starts.
struct DevRun {
  uint32_t entry;
  uint32_t pad;
  unsigned long long off;
  unsigned long long bytes;
};

// ---- work-item records ----------------------------------------------------
// Everything the control warp stages for one work item lies in one contiguous,
// 16-byte aligned record, brought into shared memory by bulk copies in a
// single round trip: the entries (step, meta word, pointer offset, dependency
// count), the prefix sums of the runs' segment counts, the runs, and the
// operand pointers of the entries' steps.  A pointer offset with PTR_GLOBAL
// set indexes the global pointer array instead (steps with many operands, or
// an item whose inline pointer area is full).
constexpr uint32_t PTR_CAP = 160;              // inline pointers per item
constexpr uint32_t SUCC_CAP = 128;             // inline successors per item
constexpr uint32_t SUCC_GLOBAL = 0xffffffffu;  // the item's successor lists stay global
constexpr uint32_t PTR_STEP_MAX = 64;          // a step with more operands keeps them global
constexpr uint32_t PTR_GLOBAL = 0x80000000u;
struct RecEnt {
  uint32_t step;
  uint32_t meta;
  uint32_t poff;    // inline pointer index, or PTR_GLOBAL | global pointer index
  uint32_t indeg;   // dependency count of the step
};
struct DevItem {
  uint32_t rec;     // record offset in 16-byte units
  uint32_t nent;
  uint32_t nrun;
  uint32_t nptr;    // inline pointers
  uint32_t nsucc;   // inline successors, or SUCC_GLOBAL
  uint32_t pad[3];
};
static_assert(sizeof(RecEnt) == 16 && sizeof(DevItem) == 32 && sizeof(DevRun) == 24, "record layout");
HICCL_HD inline uint32_t rec_ent_bytes(uint32_t nent) { return nent * 16u; }
HICCL_HD inline uint32_t rec_rpre_bytes(uint32_t nrun) { return ((nrun + 1u) * 4u + 15u) & ~15u; }
HICCL_HD inline uint32_t rec_run_bytes(uint32_t nrun) { return (nrun * 24u + 15u) & ~15u; }
HICCL_HD inline uint32_t rec_ptr_bytes(uint32_t nptr) { return (nptr * 8u + 15u) & ~15u; }
// completion section: per entry the step's completion target, then the
// offsets of the entries' successor lists (nent + 1), then the successors
HICCL_HD inline uint32_t rec_cmp_words(uint32_t nent, uint32_t nsucc) {
  return 2u * nent + 1u + (nsucc == SUCC_GLOBAL ? 0u : nsucc);
}
HICCL_HD inline uint32_t rec_cmp_bytes(uint32_t nent, uint32_t nsucc) { return (rec_cmp_words(nent, nsucc) * 4u + 15u) & ~15u; }
HICCL_HD inline uint32_t rec_bytes(const DevItem &it) {
  return rec_ent_bytes(it.nent) + rec_rpre_bytes(it.nrun) + rec_run_bytes(it.nrun) + rec_ptr_bytes(it.nptr) +
         rec_cmp_bytes(it.nent, it.nsucc);
}

// control block (device memory, zeroed at upload).  Work items are claimed
// from one ticket counter that is never reset between launches: launch e
// (from 0) makes exactly nitems + grid claims (every CTA claims until it
// draws a ticket past the last item), so ticket t belongs to launch
// t / (nitems + grid) and names item t mod (nitems + grid).  The launch index
// scales the dependency targets; no CTA does any work at exit.
struct DevCtl {
  unsigned long long ticket;   // claims so far, over all launches
  unsigned long long err;      // nonzero: abort (code << 32 | step)
};

struct DevTable {
  const unsigned char *recs;          // work-item records (16-byte aligned)
  const DevItem *items;               // [nitems] record descriptors, in ticket order
  const uint32_t *nent;               // [nsteps] entries covering the step (completion target)
  const uint32_t *succ_off;           // [nsteps + 1]
  const uint32_t *succ;               // [nedges]
  const unsigned long long *ptrs;     // [nptrs] device addresses (nsrc sources then ndst destinations per step)
  unsigned long long *dep;            // [nsteps] arrivals of predecessors (cumulative over launches)
  unsigned long long *done;           // [nsteps] finished entries (cumulative over launches)
  DevCtl *ctl;
  unsigned long long *host_err;       // mapped host word mirroring ctl->err
  unsigned long long nitems;
  unsigned long long timeout_ns;
  unsigned long long seg;             // segment bytes of this plan
  unsigned long long *trace;          // [nitems][6] timestamps, SM, first step; or null (see hiccl_get_trace)
};

enum : uint32_t { ERR_TIMEOUT = 1, ERR_BADSTEP = 2, ERR_STALL = 3 };

// ---------------------------------------------------------------------------
// host-side plan
// ---------------------------------------------------------------------------

struct Loc {
  unsigned long long addr;   // device address, or relay-arena offset when scratch
  int32_t rank;
  uint8_t scratch;
};

struct HStep {
  uint8_t kind;            // OP_COPY / OP_REDUCE
  int8_t level;            // hierarchy level crossed; -1 local
  int32_t prim;
  int32_t epoch;
  int32_t branch;
  int32_t channel;
  unsigned long long nbytes;
  uint32_t loc0;           // first Loc: nsrc sources then ndst destinations
  uint32_t nsrc;
  uint32_t ndst;
  unsigned long long slot;
  uint32_t local;          // emission index inside its piece (same tree position in every channel)
  uint32_t dtype;          // payload type of the step's communicator
  uint32_t rop;            // reduction operator (hiccl_op_t) of a reduce
  uint32_t pad3;
};

struct Prim {
  int kind;                                // 0 multicast, 1 reduction
  int op = 0;                              // hiccl_op_t of a reduction
  int root;
  std::vector<int> leaves;                 // sorted, distinct
  size_t count;
  std::vector<unsigned long long> send;    // per rank (0 = none)
  std::vector<unsigned long long> recv;
  int epoch;
};

struct DevState;   // defined by the runtime

struct Plan {
  std::vector<int> hierarchy;
  int stripe = 1, pipeline = 1;
  unsigned long long seg = SEG_BYTES;      // segment bytes (seg_bytes_of(dtype))
  std::vector<HStep> steps;                // in execution (slot) order
  std::vector<Loc> locs;
  std::vector<uint32_t> pred_off, preds;   // CSR of predecessors (by new index)
  std::vector<uint32_t> succ_off, succ;    // CSR of successors
  std::vector<DevEntry> entries;
  std::vector<uint32_t> item_off;
  std::vector<DevRun> runs;
  std::vector<uint32_t> run_off;
  std::vector<uint32_t> nent;             // entries covering each step
  unsigned long long scratch_bytes = 0;
  std::vector<unsigned long long> level_bytes;
  unsigned long long hbm_read = 0, hbm_write = 0;
  unsigned long long stages = 0, slots = 0;
  bool valid = false;
};

// Host image of the executor's read-only arrays for a plan whose relay
// offsets resolve against relay_base (hiccl_plan.cpp, build_image).
struct TableImage {
  std::vector<unsigned long long> ptrs;   // every location, resolved
  std::vector<uint32_t> indeg;            // per step
  std::vector<unsigned char> recs;        // work-item records
  std::vector<DevItem> items;             // per work item
};
void build_image(const Plan &p, unsigned long long relay_base, TableImage &im);
// bytes of TableImage::recs for plan p, without building the image
unsigned long long record_bytes(const Plan &p);

}  // namespace hiccl

struct hiccl_comm {
  int P = 0;
  hiccl_dtype_t dtype = HICCL_F32;
  int esize = 4;
  int epochs = 1;
  std::vector<hiccl::Prim> prims;
  enum State { COMPOSING, PLANNED, READY, RUNNING } state = COMPOSING;
  bool group = false;   // built by hiccl_group from other communicators' plans
  // options
  unsigned long long timeout_ns = 1000000000ull;
  int ctas_per_sm = 2;
  int threads = 256;
  unsigned long long item_bytes = 49152;   // set per payload at creation
  int order = 1;
  unsigned long long slot_items = 0;   // 0: whole rounds over the executor grid
  int trace = 0;
  int ring = 1;                       // ring(n) of Sec. 4.4; 1 = tree only
  hiccl::Plan plan;
  hiccl::DevState *dev = nullptr;
  std::string err;
};

namespace hiccl {
hiccl_status_t fail(hiccl_comm *c, hiccl_status_t st, const std::string &msg);
// Run the body of a C-ABI call so that no C++ exception leaves it: host
// memory exhaustion becomes HICCL_ERR_NOMEM, anything else HICCL_ERR_INVALID,
// with the message on `c` where there is one.
template <typename F>
hiccl_status_t guarded(hiccl_comm *c, F &&body) noexcept {
  hiccl_status_t st;
  const char *msg;
  try {
    return body();
  } catch (const std::bad_alloc &) {
    st = HICCL_ERR_NOMEM;
    msg = "out of host memory";
  } catch (...) {
    st = HICCL_ERR_INVALID;
    msg = "internal error";
  }
  try {
    return fail(c, st, msg);
  } catch (...) {
    return st;
  }
}
// factorize c's program again (hiccl_plan.cpp), keeping c's state
hiccl_status_t replan(hiccl_comm *c, const std::vector<int> &hierarchy, int stripe, int pipeline);
// runtime entry points (hiccl_runtime.cu)
hiccl_status_t dev_upload(hiccl_comm *c);
void dev_release(hiccl_comm *c);
// CTAs of an executor launch of c on the calling thread's current device
// (SMs x resident CTAs per SM for c's THREADS and CTAS_PER_SM); 0 when no
// device can be queried
unsigned long long exec_grid(const hiccl_comm &c);
}  // namespace hiccl
