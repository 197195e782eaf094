// Host side of the hierarchical collective engine: composition (paper Sec. 3),
// the factorizer (Sec. 4: striping, tree, pipelining), fence dependencies,
// race and bounds validation, the work order executed by the persistent
// kernel, and byte accounting.  Nothing here touches a GPU.
//
// Readings of the paper used by the factorizer (it is silent on them):
//  * Representative (Sec. 4.2-4.3).  A holder forwarding into a sibling
//    subgroup targets the rank at its own offset in that subgroup when that
//    rank is a leaf, else the subgroup's lowest leaf; empty subgroups are
//    pruned.  Reductions mirror multicasts.
//  * Stripe ranks (Sec. 4.3).  Branch b of s is rooted at offset (o + b) mod G
//    of the root's smallest enclosing group of G >= s ranks (o = the root's
//    offset); a primitive whose leaves all lie in that group is not striped.
//  * Pieces (Sec. 4.5).  count is cut into s*m pieces at
//    min(count, roundup(ceil(count*k/(s*m)), 16 bytes)); branch b owns pieces
//    b*m .. b*m+m-1 (its m pipeline channels).
//  * Self-delivery.  A multicast root that is a leaf with a separate
//    destination copies its piece locally in its own branch and receives the
//    other branches' pieces like any leaf; in place it takes no part.
//  * Fences (Sec. 3.3) become per-step edges from overlapping accesses.

#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "hiccl_internal.h"

using namespace hiccl;

namespace hiccl {

hiccl_status_t fail(hiccl_comm *c, hiccl_status_t st, const std::string &msg) {
  if (c) c->err = msg;
  return st;
}

// bytes of one counted unit: a value, or for FP8 a block of 128 values with
// its scale (FP8 counts are converted from values to blocks at registration)
static int esize_of(hiccl_dtype_t dt) {
  switch (dt) {
    case HICCL_F32: return 4;
    case HICCL_I32: return 4;
    case HICCL_BF16: return 2;
    case HICCL_FP8E4M3: return (int)FP8_BLOCK_BYTES;
  }
  return 0;
}

// units per piece-boundary quantum: 16 bytes of values, one FP8 block
static unsigned long long quantum_of(hiccl_dtype_t dt) {
  switch (dt) {
    case HICCL_F32: return 4;
    case HICCL_I32: return 4;
    case HICCL_BF16: return 8;
    case HICCL_FP8E4M3: return 1;
  }
  return 1;
}

// FP8 payloads are counted in values by the caller and in blocks inside
static bool to_units(hiccl_comm *c, size_t count, size_t &units) {
  if (c->dtype != HICCL_FP8E4M3) {
    units = count;
    return true;
  }
  if (count % FP8_BLOCK_ELEMS) return false;
  units = count / FP8_BLOCK_ELEMS;
  return true;
}

namespace {

// Run fn(0) .. fn(n - 1) on up to n host threads, fn(0) on the calling one;
// the share of a thread that cannot be started runs on the calling thread.
// fn must not throw.
template <typename F>
void run_parallel(int n, F &&fn) {
  std::vector<std::thread> th;
  std::vector<int> here;
  th.reserve(n);
  here.reserve(n);
  for (int t = 1; t < n; ++t) {
    try {
      th.emplace_back(fn, t);
    } catch (...) {
      here.push_back(t);
    }
  }
  fn(0);
  for (int t : here) fn(t);
  for (auto &x : th) x.join();
}

// Emits the point-to-point steps of the registered primitives (Sec. 4):
// striping, then the ring across nodes, then the tree inside them, one piece
// (branch, pipeline channel) at a time.
struct Builder {
  const hiccl_comm &c;
  std::vector<int> h;
  std::vector<long long> G;   // G[l] = prod h[l..]
  int L;
  int s, m;
  int ring = 1, lr = 0;       // ring(n) and the level of its nodes
  std::vector<HStep> steps;
  std::vector<Loc> locs;
  std::vector<std::pair<uint32_t, uint32_t>> edges;   // (pred, succ) in emission order
  unsigned long long scratch_top = 0;
  // current emission context
  int cur_prim = 0, cur_epoch = 0, cur_branch = 0, cur_channel = 0;
  uint32_t cur_local = 0, cur_relay = 0;   // steps / relays emitted in the current piece
  const Prim *p = nullptr;
  unsigned long long cur_off = 0, cur_n = 0;
  // relay buffers: allocated with ids during emission, laid out afterwards so
  // that the same relay of adjacent channels is adjacent in memory
  struct Relay {
    int prim, branch, channel;
    uint32_t local;
    unsigned long long bytes, off;
  };
  std::vector<Relay> relays;

  // the sorted leaves [b, e) of a (sub)tree, without `skip` (its holder) if present
  struct Span {
    const int *b, *e;
    int skip;
    bool empty() const { return e == b || (e - b == 1 && *b == skip); }
  };
  // per-level work lists of the tree builders, reused across calls
  struct Scratch {
    std::vector<long long> qb;
    std::vector<int> rep;
    std::vector<const int *> lo, hi;
    std::vector<Loc> locs;
    std::vector<int> prods;
    void clear() {
      qb.clear();
      rep.clear();
      lo.clear();
      hi.clear();
      locs.clear();
      prods.clear();
    }
  };
  std::vector<Scratch> scr;
  std::vector<int> grp;   // grp[l * P + r] = r / G[l + 1] (level-l subgroup of rank r)

  Builder(const hiccl_comm &comm, const std::vector<int> &hier, int stripe, int pipeline)
      : c(comm), h(hier), L((int)hier.size()), s(stripe), m(pipeline) {
    G.assign(L + 1, 1);
    for (int l = L - 1; l >= 0; --l) G[l] = G[l + 1] * h[l];
    scr.resize(L + 1);
    if ((long long)c.P * L <= (1ll << 24)) {
      grp.resize((size_t)c.P * L);
      for (int l = 0; l < L; ++l)
        for (int r = 0; r < c.P; ++r) grp[(size_t)l * c.P + r] = (int)(r / G[l + 1]);
    }
  }

  // Reserve the step, operand and edge arrays once: at the largest plans
  // (millions of steps, hundreds of millions of operands) growing them by
  // doubling costs more than the tree walks.  A piece of a primitive with n
  // leaves takes at most min(n, number of tree nodes) steps, and its operands
  // are about one per leaf plus two per step.  The estimate only sizes the
  // first allocation; a larger plan grows as usual, and a failed reservation
  // is ignored.
  void reserve_for(const std::vector<Prim> &prims) {
    unsigned long long nodes = 0;   // tree nodes of a full leaf set: sum over levels of P / G[l]
    for (int l = 0; l < L; ++l) nodes += (unsigned long long)(c.P / G[l]);
    unsigned long long ns = 0, nl = 0;
    for (const Prim &pr : prims) {
      if (!pr.count) continue;
      // at most s*m pieces, and no more than the count has quanta
      const unsigned long long q = quantum_of(c.dtype);
      const unsigned long long n = pr.leaves.size(),
                               pieces = std::min<unsigned long long>((unsigned long long)s * (unsigned long long)m,
                                                                     (pr.count + q - 1) / q);
      const unsigned long long st = std::min<unsigned long long>(n, nodes) + 2;
      ns += pieces * st;
      nl += pieces * (n + 2 * st + 4);
    }
    if (ns > 0xFFFFFFF0ull || nl > (1ull << 34)) return;   // far beyond what can be planned
    try {
      steps.reserve(ns);
      locs.reserve(nl);
      edges.reserve(ns);
    } catch (const std::bad_alloc &) {
    }
  }

  int level_of(int a, int b) const {
    if (a == b) return -1;
    if (!grp.empty()) {
      for (int l = 0; l < L; ++l)
        if (grp[(size_t)l * c.P + a] != grp[(size_t)l * c.P + b]) return l;
      return -1;
    }
    for (int l = 0; l < L; ++l)
      if (a / G[l + 1] != b / G[l + 1]) return l;
    return -1;
  }

  int emit(uint8_t kind, const Loc *srcs, uint32_t ns, const Loc *dsts, uint32_t nd, int level, const int *preds,
           uint32_t np) {
    HStep st{};
    st.kind = kind;
    st.level = (int8_t)level;
    st.prim = cur_prim;
    st.epoch = cur_epoch;
    st.branch = cur_branch;
    st.channel = cur_channel;
    st.nbytes = cur_n;
    st.local = cur_local++;
    st.dtype = (uint32_t)c.dtype;
    st.rop = p ? (uint32_t)p->op : 0u;
    st.loc0 = (uint32_t)locs.size();
    st.nsrc = ns;
    st.ndst = nd;
    locs.insert(locs.end(), srcs, srcs + ns);
    locs.insert(locs.end(), dsts, dsts + nd);
    int idx = (int)steps.size();
    steps.push_back(st);
    for (uint32_t k = 0; k < np; ++k)
      if (preds[k] >= 0) edges.emplace_back((uint32_t)preds[k], (uint32_t)idx);
    return idx;
  }
  int emit(uint8_t kind, const std::vector<Loc> &srcs, const std::vector<Loc> &dsts, int level,
           const std::vector<int> &preds) {
    return emit(kind, srcs.data(), (uint32_t)srcs.size(), dsts.data(), (uint32_t)dsts.size(), level, preds.data(),
                (uint32_t)preds.size());
  }

  Loc scratch_loc(int rank) {   // addr holds the relay id until layout_relays()
    relays.push_back(Relay{cur_prim, cur_branch, cur_channel, cur_relay++, cur_n, 0});
    return Loc{relays.size() - 1, rank, 1};
  }
  void begin_piece(int b, int ch, unsigned long long lo_bytes, unsigned long long n_bytes) {
    cur_branch = b;
    cur_channel = ch;
    cur_off = lo_bytes;
    cur_n = n_bytes;
    cur_local = 0;
    cur_relay = 0;
  }
  // place relays: the same relay of consecutive channels back to back (16-byte
  // granules), groups 256-byte aligned; then replace relay ids by offsets
  void layout_relays() {
    std::vector<uint32_t> ord(relays.size());
    std::iota(ord.begin(), ord.end(), 0u);
    std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
      const Relay &x = relays[a], &y = relays[b];
      if (x.prim != y.prim) return x.prim < y.prim;
      if (x.branch != y.branch) return x.branch < y.branch;
      if (x.local != y.local) return x.local < y.local;
      return x.channel < y.channel;
    });
    unsigned long long top = 0;
    for (size_t i = 0; i < ord.size(); ++i) {
      Relay &r = relays[ord[i]];
      const bool cont = i > 0 && relays[ord[i - 1]].prim == r.prim && relays[ord[i - 1]].branch == r.branch &&
                        relays[ord[i - 1]].local == r.local && relays[ord[i - 1]].channel + 1 == r.channel &&
                        top % 16 == 0;
      if (!cont) top = (top + 255ull) & ~255ull;
      r.off = top;
      top += r.bytes;
    }
    scratch_top = top;
    for (Loc &l : locs)
      if (l.scratch) l.addr = relays[l.addr].off;
  }
  Loc send_loc(int r) const { return Loc{p->send[r] + cur_off, r, 0}; }
  Loc recv_loc(int r) const { return Loc{p->recv[r] + cur_off, r, 0}; }
  static bool same(const Loc &a, const Loc &b) { return a.addr == b.addr && a.scratch == b.scratch; }

  // the leaves of span `sp` inside ranks [lo, hi); a span of consecutive
  // ranks (a full leaf set) is cut by arithmetic instead of searching
  static Span inside(const Span &sp, long long lo, long long hi) {
    const long long n = sp.e - sp.b;
    if (n > 0 && (long long)sp.e[-1] - sp.b[0] == n - 1) {
      const long long a = std::min(std::max(lo - sp.b[0], 0ll), n), z = std::min(std::max(hi - sp.b[0], a), n);
      return Span{sp.b + a, sp.b + z, sp.skip};
    }
    const int *a = std::lower_bound(sp.b, sp.e, (int)lo);
    const int *b = std::lower_bound(a, sp.e, (int)hi);
    return Span{a, b, sp.skip};
  }
  static bool holds(const Span &sp, long long r) {   // r is a rank of the span
    const long long n = sp.e - sp.b;
    if (n > 0 && (long long)sp.e[-1] - sp.b[0] == n - 1) return r >= sp.b[0] && r <= sp.e[-1];
    return std::binary_search(sp.b, sp.e, (int)r);
  }
  static Span span_of(const std::vector<int> &v) { return Span{v.data(), v.data() + v.size(), -1}; }
  // the representative of subgroup [qbase, qbase + sub) for `holder`: the rank
  // at the holder's offset if it is a leaf, else the lowest leaf (Sec. 4.2-4.3,
  // the g0->g6, g0->g3, g6->g9 hops of the {2,2,3} example)
  static int pick_rep(long long qbase, long long sub, int holder, const Span &ql) {
    int cand = (int)(qbase + holder % sub);
    if (cand != ql.skip && holds(ql, cand)) return cand;
    return *ql.b != ql.skip ? *ql.b : ql.b[1];
  }

  // the s branch roots of a primitive (Sec. 4.3): offsets o, o+1, ..., o+s-1
  // (mod G) of the root's smallest enclosing group of G >= s ranks; a primitive
  // whose leaves all lie in that group is not striped
  std::vector<int> stripe_ranks(int root, const std::vector<int> &leaves) const {
    if (s == 1) return {root};
    int l = L;
    while (G[l] < s) --l;   // smallest enclosing group with >= s ranks
    long long g = G[l];
    long long base = root - root % g, o = root % g;
    bool all_inside = true;
    for (int r : leaves)
      if (r < base || r >= base + g) { all_inside = false; break; }
    if (all_inside) return {root};
    std::vector<int> ks(s);
    for (int b = 0; b < s; ++b) ks[b] = (int)(base + (o + b) % g);
    return ks;
  }

  // ---- multicast tree: deliver from `holder` to every rank of `leaves` ---------
  // One hop per level from the holder to the representatives of its sibling
  // subgroups (ascending), then the same inside every subgroup (Sec. 4.2).
  void mcast_tree(int l, long long base, int holder, Loc src, int src_step, Span leaves) {
    if (l == L || leaves.empty()) return;
    const long long sub = G[l + 1];
    Scratch &S = scr[l];
    S.clear();
    if (sub == 1) {   // bottom level: every other leaf represents its own one-rank subgroup
      for (const int *i = leaves.b; i < leaves.e; ++i)
        if (*i != holder && *i != leaves.skip) S.locs.push_back(recv_loc(*i));
      if (!S.locs.empty()) emit(OP_COPY, &src, 1, S.locs.data(), (uint32_t)S.locs.size(), l, &src_step, 1);
      return;
    }
    Span own{nullptr, nullptr, leaves.skip};
    long long own_base = -1;
    for (const int *i = leaves.b; i < leaves.e;) {
      const long long qb = base + (*i - base) / sub * sub;
      const Span q = inside(Span{i, leaves.e, leaves.skip}, qb, qb + sub);
      if (holder >= qb && holder < qb + sub) {
        own = q;
        own_base = qb;
      } else if (!q.empty()) {
        S.qb.push_back(qb);
        S.rep.push_back(pick_rep(qb, sub, holder, q));
        S.lo.push_back(q.b);
        S.hi.push_back(q.e);
        S.locs.push_back(recv_loc(S.rep.back()));
      }
      i = q.e;
    }
    int hop_step = -1;
    if (!S.rep.empty()) hop_step = emit(OP_COPY, &src, 1, S.locs.data(), (uint32_t)S.locs.size(), l, &src_step, 1);
    const size_t nh = S.rep.size();
    if (own_base >= 0) mcast_tree(l + 1, own_base, holder, src, src_step, own);
    for (size_t k = 0; k < nh; ++k) {
      const Scratch &T = scr[l];   // the deeper calls use the deeper levels' lists
      const int rep = T.rep[k];
      mcast_tree(l + 1, T.qb[k], rep, recv_loc(rep), hop_step, Span{T.lo[k], T.hi[k], rep});
    }
  }

  // ---- reduction tree: fold `leaves` at `target`; returns (location, producer) ----
  // The mirror of the multicast tree (Sec. 4.2): every subgroup's partial is
  // formed at its representative, and a node folds its subgroups' partials
  // in ascending order in one reduce step.
  std::pair<Loc, int> red_tree(int l, long long base, int target, Span leaves, const Loc *out) {
    if (l == L) {
      Loc ref = send_loc(target);
      if (!out || same(*out, ref)) return {ref, -1};
      int st = emit(OP_COPY, &ref, 1, out, 1, -1, nullptr, 0);
      return {*out, st};
    }
    const long long sub = G[l + 1];
    Scratch &S = scr[l];
    S.clear();
    if (sub == 1) {   // bottom level: fold the leaves' own buffers in rank order
      if (leaves.e - leaves.b == 1 && *leaves.b == target) return red_tree(L, target, target, leaves, out);
      for (const int *i = leaves.b; i < leaves.e; ++i) {
        S.locs.push_back(send_loc(*i));
        S.prods.push_back(-1);
      }
      const size_t np = S.locs.size();
      Loc o = out ? *out : scratch_loc(target);
      int st = emit(np > 1 ? OP_REDUCE : OP_COPY, S.locs.data(), (uint32_t)np, &o, 1, l, S.prods.data(), (uint32_t)np);
      return {o, st};
    }
    for (const int *i = leaves.b; i < leaves.e;) {
      const long long qb = base + (*i - base) / sub * sub;
      const Span q = inside(Span{i, leaves.e, -1}, qb, qb + sub);
      S.qb.push_back(qb);
      S.rep.push_back((target >= qb && target < qb + sub) ? target : pick_rep(qb, sub, target, q));
      S.lo.push_back(q.b);
      S.hi.push_back(q.e);
      i = q.e;
    }
    if (S.rep.size() == 1 && S.rep[0] == target)
      return red_tree(l + 1, S.qb[0], target, Span{S.lo[0], S.hi[0], -1}, out);
    const size_t np = S.rep.size();
    for (size_t k = 0; k < np; ++k) {
      auto r = red_tree(l + 1, scr[l].qb[k], scr[l].rep[k], Span{scr[l].lo[k], scr[l].hi[k], -1}, nullptr);
      scr[l].locs.push_back(r.first);
      scr[l].prods.push_back(r.second);
    }
    Loc o = out ? *out : scratch_loc(target);
    const Scratch &T = scr[l];
    int st = emit(np > 1 ? OP_REDUCE : OP_COPY, T.locs.data(), (uint32_t)np, &o, 1, l, T.prods.data(), (uint32_t)np);
    return {o, st};
  }

  // ---- ring across the nodes of level lr (Sec. 4.4), tree inside them ----------
  // chain order: the holder's node first, then ascending node index, cyclically
  Span node_leaves(long long a, const Span &leaves) const { return inside(leaves, a * G[lr], (a + 1) * G[lr]); }

  void mcast_ring(int holder, Loc src, int src_step, Span leaves) {
    if (ring == 1) {
      mcast_tree(0, 0, holder, src, src_step, leaves);
      return;
    }
    const long long N = G[lr], a0 = holder / N;
    mcast_tree(lr, a0 * N, holder, src, src_step, node_leaves(a0, leaves));
    for (int i = 1; i < ring; ++i) {
      const long long a = (a0 + i) % ring;
      const Span nl = node_leaves(a, leaves);
      if (nl.empty()) continue;
      const int e = pick_rep(a * N, N, holder, nl);
      const Loc d = recv_loc(e);
      const int hop = emit(OP_COPY, &src, 1, &d, 1, level_of(holder, e), &src_step, 1);
      mcast_tree(lr, a * N, e, d, hop, Span{nl.b, nl.e, e});
      holder = e;
      src = d;
      src_step = hop;
    }
  }

  // the fold along the chain: the last node's tree fold travels back, each
  // earlier entry rank folds its node's partials and then the incoming one
  std::pair<Loc, int> red_ring(int target, Span leaves, const Loc *out) {
    if (ring == 1) return red_tree(0, 0, target, leaves, out);
    const long long N = G[lr], a0 = target / N;
    struct Node { long long a; Span nl; int e; };
    std::vector<Node> chain;
    int prev = target;
    for (int i = 0; i < ring; ++i) {
      const long long a = (a0 + i) % ring;
      const Span nl = node_leaves(a, leaves);
      if (nl.empty()) continue;
      const int e = a == a0 ? target : pick_rep(a * N, N, prev, nl);
      chain.push_back(Node{a, nl, e});
      prev = e;
    }
    std::pair<Loc, int> inc{};
    int inc_rank = -1;
    for (size_t k = chain.size(); k-- > 0;) {
      const Node &nd = chain[k];
      const Loc *o = (k == 0 && nd.e == target) ? out : nullptr;
      if (inc_rank < 0) {
        inc = red_tree(lr, nd.a * N, nd.e, nd.nl, o);
      } else {
        std::vector<Loc> ins;
        std::vector<int> producers;
        int lvl = level_of(inc_rank, nd.e);
        if (lr == L) {
          ins.push_back(send_loc(nd.e));
        } else {
          const long long sub = G[lr + 1];
          for (int q = 0; q < h[lr]; ++q) {
            const long long qb = nd.a * N + q * sub;
            const Span ql = inside(nd.nl, qb, qb + sub);
            if (ql.empty()) continue;
            const int rep = (nd.e >= qb && nd.e < qb + sub) ? nd.e : pick_rep(qb, sub, nd.e, ql);
            auto r = red_tree(lr + 1, qb, rep, ql, nullptr);
            ins.push_back(r.first);
            producers.push_back(r.second);
            const int lv = level_of(rep, nd.e);
            if (lv >= 0 && lv < lvl) lvl = lv;
          }
        }
        ins.push_back(inc.first);
        producers.push_back(inc.second);
        const Loc dst = o ? *o : scratch_loc(nd.e);
        inc = {dst, emit(OP_REDUCE, ins.data(), (uint32_t)ins.size(), &dst, 1, lvl, producers.data(),
                         (uint32_t)producers.size())};
      }
      inc_rank = nd.e;
    }
    if (inc_rank == target) return inc;
    const Loc dst = out ? *out : scratch_loc(target);
    return {dst, emit(OP_COPY, &inc.first, 1, &dst, 1, level_of(inc_rank, target), &inc.second, 1)};
  }

  // piece boundaries (Sec. 4.5): count cut into `parts` pieces at
  // min(count, roundup(ceil(count * k / parts), q)), q the 16-byte quantum
  std::vector<unsigned long long> bounds(size_t count, int parts) const {
    unsigned long long q = quantum_of(c.dtype);
    std::vector<unsigned long long> b(parts + 1);
    for (int k = 0; k <= parts; ++k) {
      unsigned __int128 num = (unsigned __int128)count * (unsigned)k;
      unsigned long long v = (unsigned long long)((num + parts - 1) / parts);
      v = (v + q - 1) / q * q;
      b[k] = std::min<unsigned long long>(v, count);
    }
    return b;
  }

  // M(root, leaves, count) (Sec. 3.1) as s striped branches of m channels:
  // stage 0 copies piece b to stripe rank k_b, which multicasts it (Sec. 4.3)
  void multicast(const Prim &pr) {
    std::vector<int> ks = stripe_ranks(pr.root, pr.leaves);
    int nb = (int)ks.size();
    auto bd = bounds(pr.count, nb * m);
    bool leaf_root = std::binary_search(pr.leaves.begin(), pr.leaves.end(), pr.root);
    bool self_copy = leaf_root && pr.recv[pr.root] != pr.send[pr.root];
    std::vector<int> others;
    for (int j : pr.leaves)
      if (j != pr.root) others.push_back(j);
    std::vector<int> branch;
    for (int b = 0; b < nb; ++b) {
      const int k = ks[b];
      if (k != pr.root) {   // the leaves of branch b: all but k (the root too, unless in place)
        branch.clear();
        for (int j : others)
          if (j != k) branch.push_back(j);
        if (self_copy) branch.insert(std::lower_bound(branch.begin(), branch.end(), pr.root), pr.root);
      }
      for (int ch = 0; ch < m; ++ch) {
        unsigned long long lo = bd[b * m + ch], hi = bd[b * m + ch + 1];
        if (hi <= lo) continue;
        begin_piece(b, ch, lo * c.esize, (hi - lo) * c.esize);
        Loc src = send_loc(pr.root);
        if (k == pr.root) {
          if (self_copy) {
            const Loc d = recv_loc(pr.root);
            emit(OP_COPY, &src, 1, &d, 1, -1, nullptr, 0);
          }
          mcast_ring(k, src, -1, span_of(others));
        } else {
          bool k_leaf = std::binary_search(pr.leaves.begin(), pr.leaves.end(), k);
          Loc dst = k_leaf ? recv_loc(k) : scratch_loc(k);
          int s0 = emit(OP_COPY, &src, 1, &dst, 1, level_of(pr.root, k), nullptr, 0);
          mcast_ring(k, dst, s0, span_of(branch));
        }
      }
    }
  }

  // R(leaves, root, count) (Sec. 3.1), the mirror: piece b is reduced at
  // stripe rank k_b and copied to the root (Sec. 4.3)
  void reduction(const Prim &pr) {
    std::vector<int> ks = stripe_ranks(pr.root, pr.leaves);
    int nb = (int)ks.size();
    auto bd = bounds(pr.count, nb * m);
    for (int b = 0; b < nb; ++b) {
      for (int ch = 0; ch < m; ++ch) {
        unsigned long long lo = bd[b * m + ch], hi = bd[b * m + ch + 1];
        if (hi <= lo) continue;
        begin_piece(b, ch, lo * c.esize, (hi - lo) * c.esize);
        int k = ks[b];
        Loc fin = recv_loc(pr.root);
        if (k == pr.root) {
          red_ring(k, span_of(pr.leaves), &fin);
        } else {
          auto r = red_ring(k, span_of(pr.leaves), nullptr);
          emit(OP_COPY, &r.first, 1, &fin, 1, level_of(k, pr.root), &r.second, 1);
        }
      }
    }
  }
};

struct Access {
  unsigned long long lo, hi;
  uint32_t step;
  bool write;
};

struct Range {
  unsigned long long lo, hi;
  int prim;
  bool write;
  int rank = -1;   // owner of the buffer
};

// user-buffer ranges a primitive reads and writes (an exact in-place root
// takes no part)
void prim_ranges(const hiccl_comm &c, int i, std::vector<Range> &rs) {
  const Prim &p = c.prims[i];
  if (p.count == 0) return;
  unsigned long long n = (unsigned long long)p.count * c.esize;
  if (p.kind == 0) {
    rs.push_back(Range{p.send[p.root], p.send[p.root] + n, i, false, p.root});
    for (int j : p.leaves) {
      if (j == p.root && p.recv[j] == p.send[p.root]) continue;
      rs.push_back(Range{p.recv[j], p.recv[j] + n, i, true, j});
    }
  } else {
    for (int j : p.leaves) {
      if (j == p.root && p.send[j] == p.recv[p.root]) continue;   // exact in place
      rs.push_back(Range{p.send[j], p.send[j] + n, i, false, j});
    }
    rs.push_back(Range{p.recv[p.root], p.recv[p.root] + n, i, true, p.root});
  }
}

// sorted by lo, with prefix maxima of hi: every range overlapping [lo, hi)
// is found by a binary search on hi and a backward scan
struct RangeIndex {
  std::vector<Range> r;
  std::vector<unsigned long long> pmax;
  void build() {
    std::sort(r.begin(), r.end(), [](const Range &a, const Range &b) { return a.lo < b.lo; });
    pmax.resize(r.size());
    for (size_t k = 0; k < r.size(); ++k) pmax[k] = std::max(r[k].hi, k ? pmax[k - 1] : 0ull);
  }
  template <typename F>
  void overlaps(unsigned long long lo, unsigned long long hi, F f) const {
    size_t k = std::lower_bound(r.begin(), r.end(), hi, [](const Range &x, unsigned long long v) { return x.lo < v; }) -
               r.begin();
    while (k > 0) {
      --k;
      if (pmax[k] <= lo) break;
      if (r[k].hi > lo && r[k].lo < hi) f(r[k]);
    }
  }
};

// fence dependencies (Sec. 3.3): edges from earlier-epoch steps to the steps
// of epoch e whose user-buffer accesses conflict with theirs.  Only the
// "hot" byte ranges, where a primitive of epoch e and an earlier one conflict
// (one of them writes), can hold conflicting step accesses; step accesses
// outside them are skipped before the step-level matching.
void fence_edges(Builder &B, const std::vector<uint32_t> &epoch_first) {
  const hiccl_comm &c = B.c;
  struct Span {
    unsigned long long lo, hi;
  };
  std::vector<Span> hot;
  std::vector<std::vector<int>> hot_ranks(c.prims.size());   // per primitive, ranks with hot ranges
  auto in_hot = [&](unsigned long long lo, unsigned long long hi) {
    auto it = std::upper_bound(hot.begin(), hot.end(), lo, [](unsigned long long v, const Span &x) { return v < x.hi; });
    return it != hot.end() && it->lo < hi;
  };
  auto collect = [&](uint32_t s, std::vector<Access> &out) {
    const HStep &st = B.steps[s];
    const std::vector<int> &hr = hot_ranks[st.prim];
    if (hr.empty()) return;
    for (uint32_t k = 0; k < st.nsrc + st.ndst; ++k) {
      const Loc &l = B.locs[st.loc0 + k];
      if (l.scratch || std::find(hr.begin(), hr.end(), l.rank) == hr.end() || !in_hot(l.addr, l.addr + st.nbytes))
        continue;
      out.push_back(Access{l.addr, l.addr + st.nbytes, s, k >= st.nsrc});
    }
  };
  for (size_t e = 1; e + 1 < epoch_first.size(); ++e) {
    uint32_t first = epoch_first[e], end = epoch_first[e + 1];
    if (first == end || first == 0) continue;
    // conflicting primitive ranges of epoch e against all earlier epochs
    RangeIndex earlier;
    std::vector<Range> mine;
    for (size_t i = 0; i < c.prims.size(); ++i) {
      if (c.prims[i].epoch < (int)e) prim_ranges(c, (int)i, earlier.r);
      else if (c.prims[i].epoch == (int)e) prim_ranges(c, (int)i, mine);
    }
    earlier.build();
    hot.clear();
    for (auto &v : hot_ranks) v.clear();
    auto mark = [&](const Range &x) {
      std::vector<int> &v = hot_ranks[x.prim];
      if (std::find(v.begin(), v.end(), x.rank) == v.end()) v.push_back(x.rank);
    };
    for (const Range &m : mine)
      earlier.overlaps(m.lo, m.hi, [&](const Range &x) {
        if (!(m.write || x.write)) return;
        hot.push_back(Span{std::max(m.lo, x.lo), std::min(m.hi, x.hi)});
        mark(m);
        mark(x);
      });
    if (hot.empty()) continue;
    std::sort(hot.begin(), hot.end(), [](const Span &a, const Span &b) { return a.lo < b.lo; });
    size_t w = 0;
    for (size_t k = 1; k < hot.size(); ++k) {
      if (hot[k].lo <= hot[w].hi) hot[w].hi = std::max(hot[w].hi, hot[k].hi);
      else hot[++w] = hot[k];
    }
    hot.resize(w + 1);
    // step accesses inside the hot ranges
    std::vector<Access> prev;
    for (uint32_t s = 0; s < first; ++s) collect(s, prev);
    if (prev.empty()) continue;
    std::sort(prev.begin(), prev.end(), [](const Access &a, const Access &b) { return a.lo < b.lo; });
    std::vector<unsigned long long> pmax(prev.size());
    for (size_t k = 0; k < prev.size(); ++k) pmax[k] = std::max(prev[k].hi, k ? pmax[k - 1] : 0ull);
    std::vector<Access> cur;
    std::vector<uint32_t> found;
    for (uint32_t s = first; s < end; ++s) {
      cur.clear();
      collect(s, cur);
      if (cur.empty()) continue;
      found.clear();
      for (const Access &a : cur) {
        size_t k = std::lower_bound(prev.begin(), prev.end(), a.hi,
                                    [](const Access &x, unsigned long long v) { return x.lo < v; }) -
                   prev.begin();
        while (k > 0) {
          --k;
          if (pmax[k] <= a.lo) break;
          const Access &b = prev[k];
          if (b.hi > a.lo && b.lo < a.hi && (a.write || b.write)) found.push_back(b.step);
        }
      }
      std::sort(found.begin(), found.end());
      found.erase(std::unique(found.begin(), found.end()), found.end());
      for (uint32_t q : found) B.edges.emplace_back(q, s);
    }
  }
}

// race check (Sec. 3.2): primitives of one epoch must not write what another
// reads or writes; a primitive's own writes must not overlap each other or its
// reads, except an exact in-place root
bool find_race(const hiccl_comm &c, std::string &msg) {
  for (int e = 0; e < c.epochs; ++e) {
    std::vector<Range> rs;
    for (size_t i = 0; i < c.prims.size(); ++i)
      if (c.prims[i].epoch == e) prim_ranges(c, (int)i, rs);
    std::sort(rs.begin(), rs.end(), [](const Range &a, const Range &b) { return a.lo < b.lo; });
    for (size_t a = 0; a < rs.size(); ++a) {
      for (size_t b = a + 1; b < rs.size() && rs[b].lo < rs[a].hi; ++b) {
        if (!(rs[a].write || rs[b].write)) continue;
        msg = "primitives " + std::to_string(rs[a].prim) + " and " + std::to_string(rs[b].prim) +
              " overlap in epoch " + std::to_string(e);
        return true;
      }
    }
  }
  return false;
}

}  // namespace

// Work-item records (the executor's staging unit): per item its entries
// with their steps' meta words and dependency counts, the runs and the
// prefix sums of their segment counts, and the entries' operand pointers
// inline while they fit.  Meta words carry the 16-byte alignment of every
// resolved operand.
// Shape of work item i's record (rec left 0): its entries' operand pointers
// go inline, in entry order, while a step has at most PTR_STEP_MAX operands
// and the item at most PTR_CAP; its steps' successors go inline up to
// SUCC_CAP in all, else the item reads the global successor lists.
static DevItem item_shape(const Plan &p, size_t i) {
  uint32_t nptr = 0, nsucc = 0;
  for (uint32_t e = p.item_off[i]; e < p.item_off[i + 1]; ++e) {
    const uint32_t st_i = p.entries[e].step;
    const HStep &st = p.steps[st_i];
    const uint32_t np = st.nsrc + st.ndst;
    if (np <= PTR_STEP_MAX && nptr + np <= PTR_CAP) nptr += np;
    nsucc += p.succ_off[st_i + 1] - p.succ_off[st_i];
  }
  DevItem it{};
  it.nent = p.item_off[i + 1] - p.item_off[i];
  it.nrun = p.run_off[i + 1] - p.run_off[i];
  it.nptr = nptr;
  it.nsucc = nsucc <= SUCC_CAP ? nsucc : SUCC_GLOBAL;
  return it;
}

// Bytes of the work-item records of plan p (the size of TableImage::recs),
// from the record shapes without building the image.
unsigned long long record_bytes(const Plan &p) {
  const size_t NI = p.item_off.empty() ? 0 : p.item_off.size() - 1;
  unsigned long long recs = 0;
  for (size_t i = 0; i < NI; ++i) recs += rec_bytes(item_shape(p, i));
  return recs;
}

// Bytes of the device table of plan p (records, item descriptors, per-step
// targets and successor CSR, pointer array, control block), computed from
// the record shapes without building the image.
unsigned long long table_bytes(const Plan &p) {
  const size_t NI = p.item_off.empty() ? 0 : p.item_off.size() - 1;
  return record_bytes(p) + NI * sizeof(DevItem) + p.steps.size() * (4 + 4 + 16) + 4 + p.succ.size() * 4 +
         p.locs.size() * 8 + sizeof(DevCtl);
}

void build_image(const Plan &p, unsigned long long relay_base, TableImage &im) {
  const size_t N = p.steps.size(), NL = p.locs.size();
  const size_t NI = p.item_off.empty() ? 0 : p.item_off.size() - 1;
  // large plans fill the arrays on several host threads (disjoint ranges)
  const int nthr = (NI >= 32768 || NL >= (1u << 22))
                       ? (int)std::min<size_t>(8, std::max(1u, std::thread::hardware_concurrency()))
                       : 1;
  im.ptrs.resize(NL);
  run_parallel(nthr, [&](int t) {
    for (size_t k = NL * t / nthr; k < NL * (t + 1) / nthr; ++k)
      im.ptrs[k] = p.locs[k].scratch ? relay_base + p.locs[k].addr : p.locs[k].addr;
  });
  std::vector<uint32_t> meta(N);
  im.indeg.resize(N);
  run_parallel(nthr, [&](int t) {
    for (size_t i = N * t / nthr; i < N * (t + 1) / nthr; ++i) {
      const HStep &st = p.steps[i];
      im.indeg[i] = p.pred_off[i + 1] - p.pred_off[i];
      bool al = true;
      for (uint32_t k = 0; k < st.nsrc + st.ndst; ++k) al = al && (im.ptrs[st.loc0 + k] % 16 == 0);
      meta[i] = meta_pack(st.kind, st.dtype, al ? 1u : 0u, st.nsrc, st.ndst, st.rop);
    }
  });
  im.items.assign(NI, DevItem{});
  // pass 1: record sizes and offsets (the inline-pointer decision is the same
  // in both passes: entries in order while the step's operands fit)
  std::vector<unsigned long long> at(NI + 1, 0);
  for (size_t i = 0; i < NI; ++i) {
    DevItem &it = im.items[i];
    it = item_shape(p, i);
    it.rec = (uint32_t)(at[i] / 16);
    at[i + 1] = at[i] + rec_bytes(it);
  }
  im.recs.assign(at[NI], 0);
  // pass 2: fill the records in place, in parallel for large plans
  auto fill = [&](size_t i0, size_t i1) {
    for (size_t i = i0; i < i1; ++i) {
      const DevItem &it = im.items[i];
      unsigned char *q = im.recs.data() + at[i];
      RecEnt *ent = reinterpret_cast<RecEnt *>(q);
      uint32_t *rpre = reinterpret_cast<uint32_t *>(q + rec_ent_bytes(it.nent));
      DevRun *run = reinterpret_cast<DevRun *>(q + rec_ent_bytes(it.nent) + rec_rpre_bytes(it.nrun));
      unsigned long long *ptr = reinterpret_cast<unsigned long long *>(q + rec_ent_bytes(it.nent) +
                                                                       rec_rpre_bytes(it.nrun) + rec_run_bytes(it.nrun));
      uint32_t nptr = 0;
      const uint32_t e0 = p.item_off[i];
      for (uint32_t k = 0; k < it.nent; ++k) {
        const uint32_t st_i = p.entries[e0 + k].step;
        const HStep &st = p.steps[st_i];
        const uint32_t np = st.nsrc + st.ndst;
        RecEnt re{st_i, meta[st_i], PTR_GLOBAL | st.loc0, im.indeg[st_i]};
        if (np <= PTR_STEP_MAX && nptr + np <= PTR_CAP) {
          re.poff = nptr;
          std::memcpy(ptr + nptr, im.ptrs.data() + st.loc0, np * 8);
          nptr += np;
        }
        ent[k] = re;
      }
      const uint32_t r0 = p.run_off[i];
      rpre[0] = 0;
      for (uint32_t r = 0; r < it.nrun; ++r) {
        rpre[r + 1] = rpre[r] + (uint32_t)((p.runs[r0 + r].bytes + p.seg - 1) / p.seg);
        run[r] = p.runs[r0 + r];
      }
      uint32_t *cmp = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(ptr) + rec_ptr_bytes(it.nptr));
      uint32_t *soff = cmp + it.nent, *sl = cmp + 2 * it.nent + 1;
      soff[0] = 0;
      for (uint32_t k = 0; k < it.nent; ++k) {
        const uint32_t st_i = p.entries[e0 + k].step;
        cmp[k] = p.nent[st_i];
        const uint32_t a = p.succ_off[st_i], z = p.succ_off[st_i + 1];
        if (it.nsucc != SUCC_GLOBAL) {
          for (uint32_t q = a; q < z; ++q) sl[soff[k] + (q - a)] = p.succ[q];
          soff[k + 1] = soff[k] + (z - a);
        } else {
          soff[k + 1] = 0;
        }
      }
    }
  };
  run_parallel(nthr, [&](int t) { fill(NI * t / nthr, NI * (t + 1) / nthr); });
}


// Consistency of a finished plan, checked before anything reaches the GPU:
// the table order is topological (every predecessor precedes its step, so
// the dependency graph has no cycle) and the successor lists mirror it;
// every user-buffer operand lies in its primitive's registered ranges and
// every relay operand inside the relay arena; the entries of each step tile
// its segments exactly once, in order; no item mixes slots (an item never
// waits on itself) or exceeds its entry bound; the runs of each item cover
// its entries' bytes.  Returns false with a message on the first violation.
bool validate_plan(const hiccl_comm &c, const Plan &p, std::string &msg) {
  const size_t N = p.steps.size();
  auto bad = [&](const std::string &m) {
    msg = m;
    return false;
  };
  if (p.pred_off.size() != N + 1 || p.succ_off.size() != N + 1 || p.nent.size() != N)
    return bad("table arrays have the wrong size");
  std::vector<uint32_t> nsucc(N, 0);
  for (size_t i = 0; i < N; ++i)
    for (uint32_t k = p.pred_off[i]; k < p.pred_off[i + 1]; ++k) {
      const uint32_t q = p.preds[k];
      if (q >= i) return bad("step " + std::to_string(i) + " depends on a later step " + std::to_string(q));
      if (p.steps[q].slot >= p.steps[i].slot)
        return bad("step " + std::to_string(i) + " is not in a later pipeline slot than its predecessor");
      ++nsucc[q];
    }
  for (size_t q = 0; q < N; ++q) {
    if (p.succ_off[q + 1] - p.succ_off[q] != nsucc[q])
      return bad("successor list of step " + std::to_string(q) + " does not mirror the predecessors");
    for (uint32_t k = p.succ_off[q]; k < p.succ_off[q + 1]; ++k)
      if (p.succ[k] <= q || p.succ[k] >= N) return bad("bad successor of step " + std::to_string(q));
  }
  for (size_t i = 0; i < N; ++i) {
    const HStep &st = p.steps[i];
    if (st.nsrc == 0 || st.ndst == 0 || (size_t)st.loc0 + st.nsrc + st.ndst > p.locs.size())
      return bad("step " + std::to_string(i) + " has bad operands");
    for (uint32_t k = 0; k < st.nsrc + st.ndst; ++k) {
      const Loc &l = p.locs[st.loc0 + k];
      if (l.scratch) {
        if (l.addr + st.nbytes > p.scratch_bytes) return bad("relay operand of step " + std::to_string(i) + " outside the arena");
        continue;
      }
      if (c.group || st.prim < 0 || (size_t)st.prim >= c.prims.size()) continue;
      const Prim &pr = c.prims[st.prim];
      const unsigned long long n = (unsigned long long)pr.count * c.esize;
      if (l.rank < 0 || l.rank >= c.P) return bad("operand of step " + std::to_string(i) + " has a bad rank");
      const unsigned long long sb = pr.send[l.rank], rb = pr.recv[l.rank];
      const bool in_send = sb && l.addr >= sb && l.addr + st.nbytes <= sb + n;
      const bool in_recv = rb && l.addr >= rb && l.addr + st.nbytes <= rb + n;
      if (!in_send && !in_recv)
        return bad("operand " + std::to_string(k) + " of step " + std::to_string(i) +
                   " lies outside its primitive's buffers");
    }
  }
  std::vector<unsigned long long> next(N, 0);
  std::vector<uint32_t> cnt(N, 0);
  for (const DevEntry &e : p.entries) {
    if (e.step >= N || e.seg_lo != next[e.step] || e.seg_hi <= e.seg_lo)
      return bad("entries of step " + std::to_string(e.step) + " do not tile its segments");
    next[e.step] = e.seg_hi;
    ++cnt[e.step];
  }
  for (size_t i = 0; i < N; ++i) {
    const unsigned long long nseg = (p.steps[i].nbytes + p.seg - 1) / p.seg;
    if (next[i] != nseg || cnt[i] != p.nent[i])
      return bad("entries of step " + std::to_string(i) + " do not cover it exactly once");
  }
  if (p.item_off.empty() || p.item_off.back() != p.entries.size() || p.run_off.size() != p.item_off.size())
    return bad("item offsets do not cover the entries");
  for (size_t it = 0; it + 1 < p.item_off.size(); ++it) {
    const uint32_t e0 = p.item_off[it], e1 = p.item_off[it + 1];
    if (e1 <= e0 || e1 - e0 > MAX_ENTRIES_PER_ITEM) return bad("item " + std::to_string(it) + " has a bad size");
    unsigned long long bytes = 0;
    for (uint32_t e = e0; e < e1; ++e) {
      const DevEntry &en = p.entries[e];
      if (p.steps[en.step].slot != p.steps[p.entries[e0].step].slot)
        return bad("item " + std::to_string(it) + " mixes pipeline slots");
      bytes += std::min<unsigned long long>(p.steps[en.step].nbytes, (unsigned long long)en.seg_hi * p.seg) -
               (unsigned long long)en.seg_lo * p.seg;
    }
    unsigned long long rbytes = 0;
    for (uint32_t r = p.run_off[it]; r < p.run_off[it + 1]; ++r) {
      if (p.runs[r].entry >= e1 - e0) return bad("run of item " + std::to_string(it) + " names a bad entry");
      rbytes += p.runs[r].bytes;
    }
    if (rbytes != bytes) return bad("runs of item " + std::to_string(it) + " do not cover its entries");
  }
  return true;
}

static hiccl_status_t build_plan(hiccl_comm *c, const int *hierarchy, int nlevels, int stripe,
                                 int pipeline) {
  if (!hierarchy || nlevels < 1 || nlevels > 64) return fail(c, HICCL_ERR_INVALID, "bad hierarchy");
  std::vector<int> h(hierarchy, hierarchy + nlevels);
  long long prod = 1;
  for (int f : h) {
    if (f < 1) return fail(c, HICCL_ERR_INVALID, "hierarchy factors must be >= 1");
    prod *= f;
    if (prod > (1ll << 30)) return fail(c, HICCL_ERR_INVALID, "hierarchy product too large");
  }
  if (prod != c->P)
    return fail(c, HICCL_ERR_INVALID, "product of hierarchy (" + std::to_string(prod) +
                                          ") != nranks (" + std::to_string(c->P) + ")");
  if (stripe < 1 || stripe > c->P) return fail(c, HICCL_ERR_INVALID, "stripe must be in [1, nranks]");
  if (pipeline < 1 || pipeline > 65536) return fail(c, HICCL_ERR_INVALID, "pipeline must be in [1, 65536]");
  // ring(n): its nodes must be the groups of one level (Sec. 4.4)
  int ring_lvl = -1;
  {
    long long g = c->P;
    for (int l = 0; l <= nlevels; ++l) {
      if (g * c->ring == c->P) { ring_lvl = l; break; }
      if (l < nlevels) g /= h[l];
    }
  }
  if (ring_lvl < 0)
    return fail(c, HICCL_ERR_INVALID, "ring(" + std::to_string(c->ring) +
                                          ") is not a product of the top hierarchy factors");
  if (c->ring > 1 && stripe > c->P / c->ring)
    return fail(c, HICCL_ERR_INVALID, "with a ring the stripe may not exceed the node size");
  std::string msg;
  if (find_race(*c, msg)) return fail(c, HICCL_ERR_RACE, "race: " + msg);

  Builder B(*c, h, stripe, pipeline);
  B.ring = c->ring;
  B.lr = ring_lvl;
  B.reserve_for(c->prims);
  std::vector<uint32_t> epoch_first(c->epochs + 1, 0);
  int e_seen = 0;
  for (size_t i = 0; i < c->prims.size(); ++i) {
    const Prim &p = c->prims[i];
    while (e_seen < p.epoch) epoch_first[++e_seen] = (uint32_t)B.steps.size();
    if (p.count == 0) continue;
    B.p = &p;
    B.cur_prim = (int)i;
    B.cur_epoch = p.epoch;
    if (p.kind == 0) B.multicast(p);
    else B.reduction(p);
    if (B.steps.size() > 0xFFFFFFF0ull) return fail(c, HICCL_ERR_NOMEM, "too many steps");
  }
  while (e_seen < c->epochs) epoch_first[++e_seen] = (uint32_t)B.steps.size();
  B.layout_relays();
  fence_edges(B, epoch_first);

  const size_t N = B.steps.size();
  for (const HStep &st : B.steps)
    if (st.nsrc > MAX_FANIN || st.ndst > MAX_FANIN)
      return fail(c, HICCL_ERR_UNSUPPORTED, "a step has more than 1024 inputs or outputs");

  // (every operand lying in its primitive's buffers or in the relay arena is
  // checked with the rest of the plan at the end)

  // predecessor lists in emission order (every edge points backwards)
  std::vector<uint32_t> pcount(N + 1, 0);
  std::sort(B.edges.begin(), B.edges.end(), [](auto &a, auto &b) {
    return a.second != b.second ? a.second < b.second : a.first < b.first;
  });
  B.edges.erase(std::unique(B.edges.begin(), B.edges.end()), B.edges.end());
  for (auto &e : B.edges) {
    if (e.first >= e.second) return fail(c, HICCL_ERR_INVALID, "internal: forward dependency");
    pcount[e.second + 1]++;
  }
  for (size_t i = 0; i < N; ++i) pcount[i + 1] += pcount[i];

  // stage depth and pipeline slot: a step runs one slot after its latest
  // predecessor, and channel c of a branch starts at slot c (Sec. 4.5, Fig. 7)
  std::vector<unsigned long long> depth(N, 0), slot(N, 0);
  unsigned long long maxdepth = 0, maxslot = 0;
  for (size_t i = 0; i < N; ++i) {
    unsigned long long d = 0, sl = 0;
    for (uint32_t k = pcount[i]; k < pcount[i + 1]; ++k) {
      uint32_t q = B.edges[k].first;
      d = std::max(d, depth[q] + 1);
      sl = std::max(sl, slot[q] + 1);
    }
    depth[i] = d;
    slot[i] = c->order == 0 ? std::max<unsigned long long>(sl, (unsigned long long)B.steps[i].channel) : d;
    maxdepth = std::max(maxdepth, d);
    maxslot = std::max(maxslot, slot[i]);
  }

  // data-path class of a step (see the executor): 0 = copy whose operands
  // are all 16-byte aligned, moved by bulk asynchronous copies; 1 = aligned
  // reduce of at most TMA_MAX_FANIN inputs, bulk-loaded into shared memory and
  // folded there; 2 = anything else, moved by vector loads and stores.  Relay
  // buffers are 256-byte aligned.
  std::vector<uint8_t> klass(N, 2);
  for (size_t i = 0; i < N; ++i) {
    const HStep &st = B.steps[i];
    bool al = true;
    for (uint32_t k = 0; k < st.nsrc + st.ndst; ++k) {
      const Loc &l = B.locs[st.loc0 + k];
      al = al && (l.scratch || l.addr % 16 == 0);
    }
    if (!al) continue;
    if (st.kind == OP_COPY) klass[i] = 0;
    else if (st.nsrc <= TMA_MAX_FANIN) klass[i] = 1;
  }

  // execution order: by slot, then data-path class, then emission order; a
  // slot has no internal dependencies, so any order inside it is valid
  std::vector<uint32_t> order(N);
  std::iota(order.begin(), order.end(), 0u);
  // (inside a slot: primitive, branch, tree position, channel -- so the same
  // step of adjacent channels is adjacent and can move as one range).  The
  // key identifies a step, so no two compare equal; it is packed into two
  // words when every field fits its bits, else compared field by field.
  {
    unsigned long long mprim = 0, mbranch = 0, mlocal = 0, mchan = 0;
    for (const HStep &st : B.steps) {
      mprim = std::max<unsigned long long>(mprim, (unsigned)st.prim);
      mbranch = std::max<unsigned long long>(mbranch, (unsigned)st.branch);
      mlocal = std::max<unsigned long long>(mlocal, st.local);
      mchan = std::max<unsigned long long>(mchan, (unsigned)st.channel);
    }
    if (maxslot < (1ull << 30) && mprim < (1ull << 32) && mbranch < (1ull << 30) && mlocal < (1ull << 18) &&
        mchan < (1ull << 16)) {
      struct Key {
        unsigned long long hi, lo;
        uint32_t idx;
      };
      std::vector<Key> keys(N);
      for (size_t i = 0; i < N; ++i) {
        const HStep &st = B.steps[i];
        keys[i] = Key{(slot[i] << 34) | ((unsigned long long)klass[i] << 32) | (unsigned)st.prim,
                      ((unsigned long long)(unsigned)st.branch << 34) | ((unsigned long long)st.local << 16) |
                          (unsigned)st.channel,
                      (uint32_t)i};
      }
      std::sort(keys.begin(), keys.end(),
                [](const Key &a, const Key &b) { return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo; });
      for (size_t k = 0; k < N; ++k) order[k] = keys[k].idx;
    } else {
      std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        if (slot[a] != slot[b]) return slot[a] < slot[b];
        if (klass[a] != klass[b]) return klass[a] < klass[b];
        const HStep &x = B.steps[a], &y = B.steps[b];
        if (x.prim != y.prim) return x.prim < y.prim;
        if (x.branch != y.branch) return x.branch < y.branch;
        if (x.local != y.local) return x.local < y.local;
        return x.channel < y.channel;
      });
    }
  }
  std::vector<uint32_t> pos(N);
  for (size_t k = 0; k < N; ++k) pos[order[k]] = (uint32_t)k;

  Plan plan;
  plan.hierarchy = h;
  plan.stripe = stripe;
  plan.pipeline = pipeline;
  plan.steps.resize(N);
  for (size_t k = 0; k < N; ++k) {
    plan.steps[k] = B.steps[order[k]];
    plan.steps[k].slot = slot[order[k]];
  }
  // operands stay in emission order: a step names its own with loc0
  plan.locs = std::move(B.locs);
  // predecessor and successor CSR in the new numbering
  plan.pred_off.assign(N + 1, 0);
  plan.succ_off.assign(N + 1, 0);
  for (auto &e : B.edges) {
    plan.pred_off[pos[e.second] + 1]++;
    plan.succ_off[pos[e.first] + 1]++;
  }
  for (size_t i = 0; i < N; ++i) {
    plan.pred_off[i + 1] += plan.pred_off[i];
    plan.succ_off[i + 1] += plan.succ_off[i];
  }
  plan.preds.resize(B.edges.size());
  plan.succ.resize(B.edges.size());
  {
    std::vector<uint32_t> pf(plan.pred_off.begin(), plan.pred_off.end() - 1);
    std::vector<uint32_t> sf(plan.succ_off.begin(), plan.succ_off.end() - 1);
    for (auto &e : B.edges) {
      uint32_t a = pos[e.first], b = pos[e.second];
      plan.preds[pf[b]++] = a;
      plan.succ[sf[a]++] = b;
    }
    for (size_t i = 0; i < N; ++i) {
      std::sort(plan.preds.begin() + plan.pred_off[i], plan.preds.begin() + plan.pred_off[i + 1]);
      std::sort(plan.succ.begin() + plan.succ_off[i], plan.succ.begin() + plan.succ_off[i + 1]);
    }
  }

  // work items: consecutive steps of one slot (so no item depends on itself)
  // and one data-path class, cut into runs of at most `cap` segment bytes and
  // MAX_ENTRIES_PER_ITEM steps.  A slot of S bytes is spread over about D
  // items (cap = S / D in whole segments, at most ITEM_BYTES): by default a
  // slot under SMALL_SLOT_BYTES over exactly the executor's grid, G CTAs, so
  // that a short slot -- the early levels of a tree, short but on the
  // critical path -- runs as one round of items on every CTA, and a larger
  // slot over LARGE_SLOT_ITEMS; SLOT_ITEMS > 0 sets D for every slot.
  const unsigned long long SEGB = seg_bytes_of((uint32_t)c->dtype);
  plan.seg = SEGB;
  unsigned long long G = c->slot_items ? 0 : exec_grid(*c);
  if (!c->slot_items && !G) G = DEFAULT_GRID;
  std::vector<unsigned long long> slot_bytes(N ? plan.steps.back().slot + 1 : 0, 0);
  for (const HStep &st : plan.steps) slot_bytes[st.slot] += st.nbytes;
  auto slot_cap = [&](unsigned long long sl) {
    const unsigned long long D = c->slot_items ? c->slot_items
                                 : slot_bytes[sl] < SMALL_SLOT_BYTES ? G : LARGE_SLOT_ITEMS;
    unsigned long long v = (slot_bytes[sl] + D - 1) / D;
    v = (v + SEGB - 1) / SEGB * SEGB;
    return std::min<unsigned long long>(std::max<unsigned long long>(v, SEGB),
                                        std::max<unsigned long long>(SEGB, c->item_bytes));
  };
  unsigned long long cap = SEGB;
  plan.nent.assign(N, 0);
  plan.item_off.push_back(0);
  unsigned long long cur_segs = 0;   // bytes in the open item
  unsigned long long cur_slot = ~0ull;
  int cur_class = -1;
  auto close_item = [&]() {
    if (plan.entries.size() > plan.item_off.back()) plan.item_off.push_back((uint32_t)plan.entries.size());
    cur_segs = 0;
  };
  for (size_t k = 0; k < N; ++k) {
    const HStep &st = plan.steps[k];
    if (st.slot != cur_slot || klass[order[k]] != cur_class) {
      close_item();
      cur_slot = st.slot;
      cur_class = klass[order[k]];
      cap = slot_cap(st.slot);
    }
    unsigned long long nseg = (st.nbytes + SEGB - 1) / SEGB;
    if (nseg > 0xFFFFFFFFull) return fail(c, HICCL_ERR_UNSUPPORTED, "step too large");
    unsigned long long done = 0;
    while (done < nseg) {
      // whole segments that fit the open item (at least one)
      const unsigned long long room = cap > cur_segs ? (cap - cur_segs) / SEGB : 0;
      unsigned long long take = std::max<unsigned long long>(1, std::min(nseg - done, room));
      plan.entries.push_back(DevEntry{(uint32_t)k, (uint32_t)done, (uint32_t)(done + take), 0});
      plan.nent[k]++;
      const unsigned long long bytes = std::min(st.nbytes, (done + take) * SEGB) - done * SEGB;
      done += take;
      cur_segs += bytes;
      if (cur_segs >= cap || plan.entries.size() - plan.item_off.back() >= MAX_ENTRIES_PER_ITEM)
        close_item();
    }
  }
  close_item();

  // runs: within an item, entries whose steps have the same shape and whose
  // every operand continues the previous step's in memory move as one range
  plan.run_off.push_back(0);
  auto same_loc = [&](const Loc &a, const Loc &b, unsigned long long shift) {
    return a.scratch == b.scratch && a.addr + shift == b.addr;
  };
  for (size_t it = 0; it + 1 < plan.item_off.size(); ++it) {
    const uint32_t e0 = plan.item_off[it], e1 = plan.item_off[it + 1];
    for (uint32_t e = e0; e < e1; ++e) {
      const DevEntry &en = plan.entries[e];
      const HStep &st = plan.steps[en.step];
      const unsigned long long lo = en.seg_lo * SEGB;
      const unsigned long long hi = std::min<unsigned long long>(st.nbytes, (unsigned long long)en.seg_hi * SEGB);
      bool extend = false;
      if (e > e0 && plan.runs.size() > plan.run_off.back()) {
        const DevEntry &pe = plan.entries[e - 1];
        const HStep &ps = plan.steps[pe.step];
        if (pe.step != en.step && en.seg_lo == 0 && (unsigned long long)pe.seg_hi * SEGB >= ps.nbytes &&
            ps.kind == st.kind && ps.nsrc == st.nsrc && ps.ndst == st.ndst) {
          extend = true;
          for (uint32_t k = 0; k < st.nsrc + st.ndst && extend; ++k)
            extend = same_loc(plan.locs[ps.loc0 + k], plan.locs[st.loc0 + k], ps.nbytes);
        }
      }
      if (extend) plan.runs.back().bytes += hi - lo;
      else plan.runs.push_back(DevRun{e - e0, 0, lo, hi - lo});
    }
    plan.run_off.push_back((uint32_t)plan.runs.size());
  }

  // accounting
  plan.level_bytes.assign(h.size(), 0);
  for (const HStep &st : plan.steps) {
    const Loc *l = &plan.locs[st.loc0];
    if (st.kind == OP_COPY) {
      plan.hbm_read += st.nbytes;
      plan.hbm_write += st.nbytes * st.ndst;
      for (uint32_t k = 0; k < st.ndst; ++k) {
        int lv = B.level_of(l[0].rank, l[st.nsrc + k].rank);
        if (lv >= 0) plan.level_bytes[lv] += st.nbytes;
      }
    } else {
      plan.hbm_read += st.nbytes * st.nsrc;
      plan.hbm_write += st.nbytes;
      for (uint32_t k = 0; k < st.nsrc; ++k) {
        int lv = B.level_of(l[k].rank, l[st.nsrc].rank);
        if (lv >= 0) plan.level_bytes[lv] += st.nbytes;
      }
    }
  }
  plan.scratch_bytes = B.scratch_top;
  plan.stages = N ? maxdepth + 1 : 0;
  plan.slots = N ? maxslot + 1 : 0;
  plan.valid = true;
  {
    std::string why;
    if (!validate_plan(*c, plan, why)) return fail(c, HICCL_ERR_INVALID, "internal plan check: " + why);
  }
  c->plan = std::move(plan);
  return HICCL_OK;
}

hiccl_status_t replan(hiccl_comm *c, const std::vector<int> &hierarchy, int stripe, int pipeline) {
  return build_plan(c, hierarchy.data(), (int)hierarchy.size(), stripe, pipeline);
}

}  // namespace hiccl

// ============================================================================
// C ABI: composition, planning, queries
// ============================================================================

extern "C" {

hiccl_status_t hiccl_create(int nranks, hiccl_dtype_t dtype, hiccl_comm_t *out) {
  return guarded(nullptr, [&]() -> hiccl_status_t {
    if (!out) return HICCL_ERR_INVALID;
    *out = nullptr;
    if (nranks < 1 || nranks > (1 << 30)) return HICCL_ERR_INVALID;
    if (esize_of(dtype) == 0) return HICCL_ERR_INVALID;
    hiccl_comm *c = new (std::nothrow) hiccl_comm();
    if (!c) return HICCL_ERR_NOMEM;
    c->P = nranks;
    c->dtype = dtype;
    c->esize = esize_of(dtype);
    // measured on the executor: FP8 folds prefer larger items
    c->item_bytes = dtype == HICCL_FP8E4M3 ? 65536 : 49152;
    *out = c;
    return HICCL_OK;
  });
}

static hiccl_status_t check_leaves(hiccl_comm *c, const int *leaves, int nleaves, std::vector<int> &out,
                                   bool allow_empty) {
  out.clear();
  if (nleaves == 0 && allow_empty) return HICCL_OK;
  if (!leaves || nleaves < 1) return fail(c, HICCL_ERR_INVALID, "need at least one leaf");
  if (nleaves > c->P) return fail(c, HICCL_ERR_INVALID, "more leaves than ranks");
  out.assign(leaves, leaves + nleaves);
  for (int r : out)
    if (r < 0 || r >= c->P) return fail(c, HICCL_ERR_INVALID, "leaf rank out of range");
  std::sort(out.begin(), out.end());
  if (std::adjacent_find(out.begin(), out.end()) != out.end())
    return fail(c, HICCL_ERR_INVALID, "duplicate leaf");
  return HICCL_OK;
}

static bool aligned_elem(const hiccl_comm *c, unsigned long long a) {
  return c->dtype == HICCL_FP8E4M3 ? a % 16 == 0 : a % c->esize == 0;
}

hiccl_status_t hiccl_add_multicast(hiccl_comm_t c, const void *const *send, void *const *recv,
                                   size_t count, int root, const int *leaves, int nleaves) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "add after init");
    if (!send || !recv) return fail(c, HICCL_ERR_INVALID, "null pointer array");
    if (root < 0 || root >= c->P) return fail(c, HICCL_ERR_INVALID, "root out of range");
    Prim p;
    p.kind = 0;
    p.root = root;
    if (!to_units(c, count, p.count)) return fail(c, HICCL_ERR_INVALID, "FP8 counts must be multiples of 128");
    p.epoch = c->epochs - 1;
    hiccl_status_t st = check_leaves(c, leaves, nleaves, p.leaves, true);
    if (st != HICCL_OK) return st;
    if (p.leaves.empty()) return HICCL_OK;   // nothing to deliver
    p.send.assign(c->P, 0);
    p.recv.assign(c->P, 0);
    p.send[root] = (unsigned long long)(uintptr_t)send[root];
    for (int j : p.leaves) p.recv[j] = (unsigned long long)(uintptr_t)recv[j];
    if (count > 0) {
      if (!p.send[root]) return fail(c, HICCL_ERR_INVALID, "null send buffer at the root");
      for (int j : p.leaves)
        if (!p.recv[j]) return fail(c, HICCL_ERR_INVALID, "null recv buffer at a leaf");
      if (!aligned_elem(c, p.send[root])) return fail(c, HICCL_ERR_INVALID, "misaligned send buffer");
      for (int j : p.leaves)
        if (!aligned_elem(c, p.recv[j])) return fail(c, HICCL_ERR_INVALID, "misaligned recv buffer");
      if ((unsigned long long)p.count > (~0ull) / 256) return fail(c, HICCL_ERR_INVALID, "count too large");
    }
    c->prims.push_back(std::move(p));
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_add_reduction(hiccl_comm_t c, const void *const *send, void *const *recv,
                                   size_t count, const int *leaves, int nleaves, int root,
                                   hiccl_op_t op) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "add after init");
    if (!send || !recv) return fail(c, HICCL_ERR_INVALID, "null pointer array");
    if (op != HICCL_SUM && op != HICCL_MAX && op != HICCL_MIN && op != HICCL_LOR)
      return fail(c, HICCL_ERR_INVALID, "unknown reduction operator");
    if (op != HICCL_SUM && c->dtype == HICCL_FP8E4M3)
      return fail(c, HICCL_ERR_UNSUPPORTED, "FP8 payloads reduce with HICCL_SUM only");
    if (op == HICCL_LOR && c->dtype != HICCL_I32)
      return fail(c, HICCL_ERR_UNSUPPORTED, "HICCL_LOR needs HICCL_I32 payloads");
    if (root < 0 || root >= c->P) return fail(c, HICCL_ERR_INVALID, "root out of range");
    Prim p;
    p.kind = 1;
    p.op = (int)op;
    p.root = root;
    if (!to_units(c, count, p.count)) return fail(c, HICCL_ERR_INVALID, "FP8 counts must be multiples of 128");
    p.epoch = c->epochs - 1;
    hiccl_status_t st = check_leaves(c, leaves, nleaves, p.leaves, false);
    if (st != HICCL_OK) return st;
    p.send.assign(c->P, 0);
    p.recv.assign(c->P, 0);
    for (int j : p.leaves) p.send[j] = (unsigned long long)(uintptr_t)send[j];
    p.recv[root] = (unsigned long long)(uintptr_t)recv[root];
    if (count > 0) {
      if (!p.recv[root]) return fail(c, HICCL_ERR_INVALID, "null recv buffer at the root");
      for (int j : p.leaves)
        if (!p.send[j]) return fail(c, HICCL_ERR_INVALID, "null send buffer at a leaf");
      if (!aligned_elem(c, p.recv[root])) return fail(c, HICCL_ERR_INVALID, "misaligned recv buffer");
      for (int j : p.leaves)
        if (!aligned_elem(c, p.send[j])) return fail(c, HICCL_ERR_INVALID, "misaligned send buffer");
      if ((unsigned long long)p.count > (~0ull) / 256) return fail(c, HICCL_ERR_INVALID, "count too large");
    }
    c->prims.push_back(std::move(p));
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_add_fence(hiccl_comm_t c) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "add after init");
    c->epochs++;
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_add_collective(hiccl_comm_t c, hiccl_collective_t kind, size_t d, const void *const *send,
                                    void *const *recv, int root, hiccl_op_t op) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "add after init");
    if (!send || !recv) return fail(c, HICCL_ERR_INVALID, "null pointer array");
    const int P = c->P;
    if (root < 0 || root >= P) return fail(c, HICCL_ERR_INVALID, "root out of range");
    size_t du = 0;
    if (!to_units(c, d, du)) return fail(c, HICCL_ERR_INVALID, "FP8 counts must be multiples of 128");
    const unsigned long long cb = (unsigned long long)du * c->esize;   // bytes of one chunk
    std::vector<int> all(P), others;
    for (int r = 0; r < P; ++r) all[r] = r;
    std::vector<const void *> s(P, nullptr);
    std::vector<void *> v(P, nullptr);
    auto sa = [&](int r, unsigned long long k) { return (const void *)((const char *)send[r] + k * cb); };
    auto ra = [&](int r, unsigned long long k) { return (void *)((char *)recv[r] + k * cb); };
    auto reset = [&]() {
      std::fill(s.begin(), s.end(), nullptr);
      std::fill(v.begin(), v.end(), nullptr);
    };
    hiccl_status_t st = HICCL_OK;
    const size_t dp = d * P;
    switch (kind) {
      case HICCL_BROADCAST:
        return hiccl_add_multicast(c, send, recv, dp, root, all.data(), P);
      case HICCL_REDUCE:
        return hiccl_add_reduction(c, send, recv, dp, all.data(), P, root, op);
      case HICCL_ALLGATHER:
        for (int i = 0; i < P && st == HICCL_OK; ++i) {
          for (int r = 0; r < P; ++r) v[r] = ra(r, i);
          st = hiccl_add_multicast(c, send, v.data(), d, i, all.data(), P);
        }
        return st;
      case HICCL_REDUCESCATTER:
        for (int j = 0; j < P && st == HICCL_OK; ++j) {
          for (int r = 0; r < P; ++r) s[r] = sa(r, j);
          st = hiccl_add_reduction(c, s.data(), recv, d, all.data(), P, j, op);
        }
        return st;
      case HICCL_ALLREDUCE_SINGLE:
        for (int j = 0; j < P && st == HICCL_OK; ++j)
          st = hiccl_add_reduction(c, send, recv, dp, all.data(), P, j, op);
        return st;
      case HICCL_SCATTER:
        for (int j = 0; j < P && st == HICCL_OK; ++j) {
          reset();
          s[root] = sa(root, j);
          v[j] = recv[j];
          st = hiccl_add_reduction(c, s.data(), v.data(), d, &root, 1, j, HICCL_SUM);
        }
        return st;
      case HICCL_GATHER:
        for (int i = 0; i < P && st == HICCL_OK; ++i) {
          reset();
          s[i] = send[i];
          v[root] = ra(root, i);
          st = hiccl_add_multicast(c, s.data(), v.data(), d, i, &root, 1);
        }
        return st;
      case HICCL_ALLTOALL:
        for (int i = 0; i < P && st == HICCL_OK; ++i)
          for (int j = 0; j < P && st == HICCL_OK; ++j) {
            reset();
            s[i] = sa(i, j);
            v[j] = ra(j, i);
            st = hiccl_add_multicast(c, s.data(), v.data(), d, i, &j, 1);
          }
        return st;
      case HICCL_ALLREDUCE:
        for (int j = 0; j < P && st == HICCL_OK; ++j) {
          reset();
          for (int r = 0; r < P; ++r) s[r] = sa(r, j);
          v[j] = ra(j, j);
          st = hiccl_add_reduction(c, s.data(), v.data(), d, all.data(), P, j, op);
        }
        if (st == HICCL_OK) st = hiccl_add_fence(c);
        for (int i = 0; i < P && st == HICCL_OK; ++i) {
          others.clear();
          for (int r = 0; r < P; ++r)
            if (r != i) others.push_back(r);
          for (int r = 0; r < P; ++r) {
            s[r] = ra(r, i);
            v[r] = ra(r, i);
          }
          st = hiccl_add_multicast(c, s.data(), v.data(), d, i, others.data(), (int)others.size());
        }
        return st;
    }
    return fail(c, HICCL_ERR_INVALID, "unknown collective");
  });
}

hiccl_status_t hiccl_plan(hiccl_comm_t c, const int *hierarchy, int nlevels, int stripe, int pipeline) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state == hiccl_comm::READY || c->state == hiccl_comm::RUNNING)
      return fail(c, HICCL_ERR_STATE, "already initialized");
    hiccl_status_t st = build_plan(c, hierarchy, nlevels, stripe, pipeline);
    if (st == HICCL_OK) c->state = hiccl_comm::PLANNED;
    return st;
  });
}

hiccl_status_t hiccl_init(hiccl_comm_t c, const int *hierarchy, int nlevels, int stripe, int pipeline) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state == hiccl_comm::READY || c->state == hiccl_comm::RUNNING)
      return fail(c, HICCL_ERR_STATE, "already initialized");
    // a plan made by hiccl_plan with the same parameters is uploaded as it is:
    // nothing that feeds the factorizer can change in the planned state
    const bool same = c->state == hiccl_comm::PLANNED && c->plan.valid && hierarchy && nlevels >= 1 &&
                      c->plan.hierarchy == std::vector<int>(hierarchy, hierarchy + nlevels) &&
                      c->plan.stripe == stripe && c->plan.pipeline == pipeline;
    hiccl_status_t st = same ? HICCL_OK : build_plan(c, hierarchy, nlevels, stripe, pipeline);
    if (st != HICCL_OK) return st;
    c->state = hiccl_comm::PLANNED;
    st = dev_upload(c);
    if (st != HICCL_OK) return st;
    c->state = hiccl_comm::READY;
    return HICCL_OK;
  });
}

// The union of the planned members' tables (see hiccl_group), planned on the
// host and checked; not uploaded.  *out receives the new communicator.
static hiccl_status_t group_build(const hiccl_comm_t *comms, int n, hiccl_comm **out) {
  if (!comms || n < 1) return HICCL_ERR_INVALID;
  unsigned long long segb = 0;
  for (int i = 0; i < n; ++i) {
    if (!comms[i] || !comms[i]->plan.valid) return HICCL_ERR_STATE;
    if (segb && comms[i]->plan.seg != segb) return HICCL_ERR_UNSUPPORTED;   // FP8 with other payloads
    segb = comms[i]->plan.seg;
  }
  std::unique_ptr<hiccl_comm, void (*)(hiccl_comm_t)> owner(new (std::nothrow) hiccl_comm(), hiccl_destroy);
  hiccl_comm *g = owner.get();
  if (!g) return HICCL_ERR_NOMEM;
  g->group = true;
  g->P = comms[0]->P;
  g->dtype = comms[0]->dtype;
  g->esize = comms[0]->esize;
  g->timeout_ns = comms[0]->timeout_ns;
  g->ctas_per_sm = comms[0]->ctas_per_sm;
  g->threads = comms[0]->threads;
  Plan &P = g->plan;
  P.seg = segb;
  P.pred_off.push_back(0);
  P.succ_off.push_back(0);
  // member tables, concatenated; every member's relays move to its own range
  struct ItemRef { unsigned long long slot; uint32_t rank; int member; uint32_t item; };
  std::vector<ItemRef> items;
  std::vector<uint32_t> step_off(n), entry_off(n), run_off(n);
  unsigned long long relay_off = 0;
  for (int i = 0; i < n; ++i) {
    const Plan &q = comms[i]->plan;
    const uint32_t so = (uint32_t)P.steps.size(), lo = (uint32_t)P.locs.size();
    step_off[i] = so;
    entry_off[i] = (uint32_t)P.entries.size();
    run_off[i] = (uint32_t)P.runs.size();
    for (HStep st : q.steps) {
      st.loc0 += lo;
      P.steps.push_back(st);
    }
    for (Loc l : q.locs) {
      if (l.scratch) l.addr += relay_off;
      P.locs.push_back(l);
    }
    for (size_t k = 0; k < q.steps.size(); ++k) {
      for (uint32_t x = q.pred_off[k]; x < q.pred_off[k + 1]; ++x) P.preds.push_back(q.preds[x] + so);
      P.pred_off.push_back((uint32_t)P.preds.size());
      for (uint32_t x = q.succ_off[k]; x < q.succ_off[k + 1]; ++x) P.succ.push_back(q.succ[x] + so);
      P.succ_off.push_back((uint32_t)P.succ.size());
    }
    P.nent.insert(P.nent.end(), q.nent.begin(), q.nent.end());
    for (DevEntry e : q.entries) {
      e.step += so;
      P.entries.push_back(e);
    }
    P.runs.insert(P.runs.end(), q.runs.begin(), q.runs.end());
    // rank of each item inside its slot, for interleaving the members
    unsigned long long prev_slot = ~0ull;
    uint32_t rank = 0;
    for (size_t t = 0; t + 1 < q.item_off.size(); ++t) {
      const unsigned long long sl = q.steps[q.entries[q.item_off[t]].step].slot;
      rank = sl == prev_slot ? rank + 1 : 0;
      prev_slot = sl;
      items.push_back(ItemRef{sl, rank, i, (uint32_t)t});
    }
    relay_off = (relay_off + q.scratch_bytes + 255ull) & ~255ull;
    P.hbm_read += q.hbm_read;
    P.hbm_write += q.hbm_write;
    P.stages = std::max(P.stages, q.stages);
    P.slots = std::max(P.slots, q.slots);
  }
  P.scratch_bytes = relay_off;
  // one ticket order for all: by slot, then round-robin over the members;
  // each member keeps its own (topological) item order
  std::stable_sort(items.begin(), items.end(), [](const ItemRef &a, const ItemRef &b) {
    if (a.slot != b.slot) return a.slot < b.slot;
    if (a.rank != b.rank) return a.rank < b.rank;
    return a.member < b.member;
  });
  std::vector<DevEntry> ents;
  std::vector<DevRun> runs;
  P.item_off.assign(1, 0);
  P.run_off.assign(1, 0);
  for (const ItemRef &it : items) {
    const Plan &q = comms[it.member]->plan;
    for (uint32_t x = q.item_off[it.item]; x < q.item_off[it.item + 1]; ++x)
      ents.push_back(P.entries[entry_off[it.member] + x]);
    for (uint32_t x = q.run_off[it.item]; x < q.run_off[it.item + 1]; ++x) runs.push_back(P.runs[run_off[it.member] + x]);
    P.item_off.push_back((uint32_t)ents.size());
    P.run_off.push_back((uint32_t)runs.size());
  }
  P.entries.swap(ents);
  P.runs.swap(runs);
  P.valid = true;
  {
    std::string why;
    if (!validate_plan(*g, P, why)) return HICCL_ERR_INVALID;
  }
  g->state = hiccl_comm::PLANNED;
  *out = owner.release();
  return HICCL_OK;
}

hiccl_status_t hiccl_group(const hiccl_comm_t *comms, int n, hiccl_comm_t *out) {
  return guarded(nullptr, [&]() -> hiccl_status_t {
    if (!out) return HICCL_ERR_INVALID;
    *out = nullptr;
    hiccl_comm *g = nullptr;
    hiccl_status_t st = group_build(comms, n, &g);
    if (st != HICCL_OK) return st;
    st = dev_upload(g);
    if (st != HICCL_OK) {
      hiccl_destroy(g);
      return st;
    }
    g->state = hiccl_comm::READY;
    *out = g;
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_group_plan(const hiccl_comm_t *comms, int n, hiccl_comm_t *out) {
  return guarded(nullptr, [&]() -> hiccl_status_t {
    if (!out) return HICCL_ERR_INVALID;
    *out = nullptr;
    return group_build(comms, n, out);
  });
}

hiccl_status_t hiccl_level_bytes(hiccl_comm_t c, unsigned long long *per_level, int nlevels) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (!c->plan.valid) return fail(c, HICCL_ERR_STATE, "no plan");
    if (c->group) return fail(c, HICCL_ERR_UNSUPPORTED, "per-level bytes of a group: query its members");
    if (!per_level || nlevels != (int)c->plan.level_bytes.size())
      return fail(c, HICCL_ERR_INVALID, "nlevels must equal the hierarchy's");
    for (int l = 0; l < nlevels; ++l) per_level[l] = c->plan.level_bytes[l];
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_hbm_bytes(hiccl_comm_t c, unsigned long long *rd, unsigned long long *wr) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (!c->plan.valid) return fail(c, HICCL_ERR_STATE, "no plan");
    if (rd) *rd = c->plan.hbm_read;
    if (wr) *wr = c->plan.hbm_write;
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_validate(hiccl_comm_t c) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (!c->plan.valid) return fail(c, HICCL_ERR_STATE, "no plan");
    std::string why;
    if (!validate_plan(*c, c->plan, why)) return fail(c, HICCL_ERR_INVALID, "plan check: " + why);
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_debug_image(hiccl_comm_t c, void *recs, size_t recs_capacity, size_t *recs_bytes,
                                 void *items, size_t items_capacity, size_t *nitems) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (!c->plan.valid) return fail(c, HICCL_ERR_STATE, "not planned");
    TableImage im;
    build_image(c->plan, 0, im);
    if (recs_bytes) *recs_bytes = im.recs.size();
    if (nitems) *nitems = im.items.size();
    if (recs && recs_capacity >= im.recs.size()) std::memcpy(recs, im.recs.data(), im.recs.size());
    if (items && items_capacity >= im.items.size() * sizeof(DevItem))
      std::memcpy(items, im.items.data(), im.items.size() * sizeof(DevItem));
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_debug_corrupt(hiccl_comm_t c, int what) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    if (c->state != hiccl_comm::PLANNED || !c->plan.valid)
      return fail(c, HICCL_ERR_STATE, "needs a planned communicator that is not uploaded");
    Plan &p = c->plan;
    const size_t N = p.steps.size();
    switch (what) {
      case 0: {   // a dependency on a later step: a cycle in the dependency graph
        for (size_t i = 0; i + 1 < N; ++i)
          if (p.pred_off[i + 1] > p.pred_off[i]) {
            p.preds[p.pred_off[i]] = (uint32_t)(N - 1);
            return HICCL_OK;
          }
        return fail(c, HICCL_ERR_INVALID, "no step with a predecessor");
      }
      case 1: {   // a user-buffer operand moved out of its primitive's buffers
        for (const HStep &st : p.steps)
          for (uint32_t k = 0; k < st.nsrc + st.ndst; ++k)
            if (!p.locs[st.loc0 + k].scratch) {
              p.locs[st.loc0 + k].addr += (unsigned long long)c->prims[st.prim].count * c->esize + 4096;
              return HICCL_OK;
            }
        return fail(c, HICCL_ERR_INVALID, "no user operand");
      }
      case 2: {   // the last entry of a step dropped: segments left uncovered
        if (p.entries.empty()) return fail(c, HICCL_ERR_INVALID, "no entries");
        p.entries.back().seg_hi = p.entries.back().seg_lo;
        return HICCL_OK;
      }
      default:
        return fail(c, HICCL_ERR_INVALID, "unknown corruption");
    }
  });
}

hiccl_status_t hiccl_plan_info(hiccl_comm_t c, hiccl_plan_info_t *out) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c || !out) return HICCL_ERR_INVALID;
    if (!c->plan.valid) return fail(c, HICCL_ERR_STATE, "no plan");
    const Plan &p = c->plan;
    std::memset(out, 0, sizeof(*out));
    out->steps = p.steps.size();
    for (const HStep &st : p.steps) (st.kind == OP_COPY ? out->copy_steps : out->reduce_steps)++;
    out->items = p.item_off.size() - 1;
    out->edges = p.succ.size();
    out->stages = p.stages;
    out->slots = p.slots;
    out->runs = p.runs.size();
    out->scratch_bytes = p.scratch_bytes;
    out->table_bytes = table_bytes(p);
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_get_step(hiccl_comm_t c, unsigned long long index, hiccl_step_desc_t *d,
                              unsigned long long *src_addr, int *src_scratch, int *src_rank,
                              unsigned long long *dst_addr, int *dst_scratch, int *dst_rank,
                              unsigned long long *preds) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c || !d) return HICCL_ERR_INVALID;
    if (!c->plan.valid) return fail(c, HICCL_ERR_STATE, "no plan");
    const Plan &p = c->plan;
    if (index >= p.steps.size()) return fail(c, HICCL_ERR_INVALID, "step index out of range");
    const HStep &st = p.steps[index];
    d->kind = st.kind;
    d->level = st.level;
    d->nsrc = (int)st.nsrc;
    d->ndst = (int)st.ndst;
    d->npreds = (int)(p.pred_off[index + 1] - p.pred_off[index]);
    d->prim = st.prim;
    d->branch = st.branch;
    d->channel = st.channel;
    d->op = st.kind == 1 ? (int)st.rop : 0;
    d->reserved = 0;
    d->nbytes = st.nbytes;
    d->slot = st.slot;
    for (uint32_t k = 0; k < st.nsrc; ++k) {
      const Loc &l = p.locs[st.loc0 + k];
      if (src_addr) src_addr[k] = l.addr;
      if (src_scratch) src_scratch[k] = l.scratch;
      if (src_rank) src_rank[k] = l.rank;
    }
    for (uint32_t k = 0; k < st.ndst; ++k) {
      const Loc &l = p.locs[st.loc0 + st.nsrc + k];
      if (dst_addr) dst_addr[k] = l.addr;
      if (dst_scratch) dst_scratch[k] = l.scratch;
      if (dst_rank) dst_rank[k] = l.rank;
    }
    if (preds)
      for (uint32_t k = p.pred_off[index]; k < p.pred_off[index + 1]; ++k) preds[k - p.pred_off[index]] = p.preds[k];
    return HICCL_OK;
  });
}

hiccl_status_t hiccl_set_option(hiccl_comm_t c, hiccl_option_t opt, long long value) {
  return guarded(c, [&]() -> hiccl_status_t {
    if (!c) return HICCL_ERR_INVALID;
    switch (opt) {
      case HICCL_OPT_TIMEOUT_NS:
        if (value < 1000) return fail(c, HICCL_ERR_INVALID, "timeout below 1 us");
        c->timeout_ns = (unsigned long long)value;
        return HICCL_OK;
      case HICCL_OPT_CTAS_PER_SM:
        if (value < 1 || value > 32) return fail(c, HICCL_ERR_INVALID, "ctas per SM must be in [1, 32]");
        c->ctas_per_sm = (int)value;
        return HICCL_OK;
      case HICCL_OPT_THREADS:
        if (value != 128 && value != 256 && value != 512)
          return fail(c, HICCL_ERR_INVALID, "threads per CTA must be 128, 256 or 512");
        c->threads = (int)value;
        return HICCL_OK;
      case HICCL_OPT_TRACE:
        if (c->state != hiccl_comm::COMPOSING && c->state != hiccl_comm::PLANNED)
          return fail(c, HICCL_ERR_STATE, "set before hiccl_init");
        c->trace = value ? 1 : 0;
        return HICCL_OK;
      case HICCL_OPT_SLOT_ITEMS:
        if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "set before planning");
        if (value < 1 || value > (1ll << 24)) return fail(c, HICCL_ERR_INVALID, "slot items out of range");
        c->slot_items = (unsigned long long)value;
        return HICCL_OK;
      case HICCL_OPT_ITEM_BYTES:
        if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "set before planning");
        if (value < (long long)SEG_BYTES || value > (1ll << 30)) return fail(c, HICCL_ERR_INVALID, "item bytes out of range");
        c->item_bytes = (unsigned long long)value;
        return HICCL_OK;
      case HICCL_OPT_RING:
        if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "set before planning");
        if (value < 1 || value > c->P) return fail(c, HICCL_ERR_INVALID, "ring must be in [1, nranks]");
        c->ring = (int)value;
        return HICCL_OK;
      case HICCL_OPT_ORDER:
        if (c->state != hiccl_comm::COMPOSING) return fail(c, HICCL_ERR_STATE, "set before planning");
        if (value != 0 && value != 1) return fail(c, HICCL_ERR_INVALID, "order must be 0 or 1");
        c->order = (int)value;
        return HICCL_OK;
    }
    return fail(c, HICCL_ERR_INVALID, "unknown option");
  });
}

const char *hiccl_last_error(hiccl_comm_t c) {
  if (!c) return "null communicator";
  return c->err.c_str();
}

void hiccl_destroy(hiccl_comm_t c) {
  if (!c) return;
  dev_release(c);
  delete c;
}

}  // extern "C"
