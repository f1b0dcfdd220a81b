// Build-time (library-load-time) generator of the recurrence programs that the
// integral kernels interpret.  For every shell-quartet class it emits:
//   * the Obara-Saika vertical recurrence (VRR) from the Boys-weighted base
//     values [00|00]^(m) to the targets [e0|f0]^(0), split into dependency
//     levels whose steps are independent (the HGP-OS tower of the paper's
//     "Computational Details": VRR on the bra, then on the ket);
//   * the accumulation of the targets into contracted accumulators (one
//     channel for plain integrals; for derivative integrals four channels
//     weighted 1, 2 alpha, 2 beta, 2 gamma -- the Gaussian derivative rule
//     d/dA g_a = 2 alpha g_{a+1} - a_x g_{a-1}, one channel per raised centre,
//     as in the paper's single-index lift, Eq. l18);
//   * the horizontal recurrence (HRR) on contracted values, bra then ket,
//     and, for derivatives, the final combination of raised and lowered blocks.
// The recurrences are standard (Obara & Saika 1986; Head-Gordon & Pople 1988);
// the code below is written from those relations.
#include <algorithm>
#include <array>
#include <map>
#include <set>
#include <stdexcept>
#include <tuple>

#include "ltjk_internal.h"

namespace ltjk {
namespace {

using Mono = std::array<int, 3>;

int mono_l(const Mono &m) { return m[0] + m[1] + m[2]; }
std::vector<Mono> monos(int l) {
  std::vector<Mono> v;
  for (int lx = l; lx >= 0; --lx)
    for (int ly = l - lx; ly >= 0; --ly) v.push_back({lx, ly, l - lx - ly});
  return v;
}
int first_dir(const Mono &m) {
  for (int i = 0; i < 3; ++i)
    if (m[i] > 0) return i;
  return -1;
}
Mono shift(Mono m, int dir, int by) {
  m[dir] += by;
  return m;
}

// Ordered set of monomials with total L in [lo, hi] -> dense index.
struct MonoSet {
  int lo, hi;
  std::map<Mono, int> idx;
  std::vector<Mono> list;
  MonoSet(int lo_, int hi_) : lo(std::max(lo_, 0)), hi(hi_) {
    for (int l = lo; l <= hi; ++l)
      for (auto &m : monos(l)) {
        idx[m] = (int)list.size();
        list.push_back(m);
      }
  }
  int size() const { return (int)list.size(); }
};

struct VrrGen {
  int ltot;
  std::map<std::tuple<Mono, Mono, int>, int> slot;  // (e, f, m) -> slot
  std::vector<int> level;                            // per slot
  std::vector<VrrInstr> instr;                       // in creation order
  std::vector<int> instr_level;
  double flops = 0;

  explicit VrrGen(int lt) : ltot(lt) {
    level.assign(ltot + 2, 0);  // slot 0 zero, 1..ltot+1 base
  }
  int get(const Mono &e, const Mono &f, int m) {
    if (mono_l(e) == 0 && mono_l(f) == 0) return 1 + m;
    auto key = std::make_tuple(e, f, m);
    auto it = slot.find(key);
    if (it != slot.end()) return it->second;
    VrrInstr in{};
    int lv;
    if (mono_l(f) > 0) {
      int i = first_dir(f);
      Mono f1 = shift(f, i, -1);
      in.kind = 1;
      in.dir = (uint8_t)i;
      in.s0 = (uint16_t)get(e, f1, m);
      in.s1 = (uint16_t)get(e, f1, m + 1);
      in.n1 = (uint8_t)f1[i];
      in.s2 = in.s3 = 0;
      if (f1[i] > 0) {
        Mono f2 = shift(f1, i, -1);
        in.s2 = (uint16_t)get(e, f2, m);
        in.s3 = (uint16_t)get(e, f2, m + 1);
      }
      in.n2 = (uint8_t)e[i];
      in.s4 = 0;
      if (e[i] > 0) in.s4 = (uint16_t)get(shift(e, i, -1), f1, m + 1);
      flops += 3 + (in.n1 ? 4 : 0) + (in.n2 ? 3 : 0);
      lv = 1 + std::max({level[in.s0], level[in.s1], level[in.s2], level[in.s3], level[in.s4]});
    } else {
      int i = first_dir(e);
      Mono e1 = shift(e, i, -1);
      in.kind = 0;
      in.dir = (uint8_t)i;
      in.s0 = (uint16_t)get(e1, f, m);
      in.s1 = (uint16_t)get(e1, f, m + 1);
      in.n1 = (uint8_t)e1[i];
      in.s2 = in.s3 = in.s4 = 0;
      in.n2 = 0;
      if (e1[i] > 0) {
        Mono e2 = shift(e1, i, -1);
        in.s2 = (uint16_t)get(e2, f, m);
        in.s3 = (uint16_t)get(e2, f, m + 1);
      }
      flops += 3 + (in.n1 ? 4 : 0);
      lv = 1 + std::max({level[in.s0], level[in.s1], level[in.s2], level[in.s3]});
    }
    int s = (int)level.size();
    if (s > 65000) throw std::runtime_error("VRR program too large");
    in.tgt = (uint16_t)s;
    level.push_back(lv);
    slot[key] = s;
    instr.push_back(in);
    instr_level.push_back(lv);
    return s;
  }
};

// HRR node: (channel, a, b, c, d); leaves are accumulators (b = d = 0).
struct HrrGen {
  const std::vector<MonoSet> *E, *F;  // per channel
  std::vector<int> acc_off;           // per channel flat offset
  int acc_total;
  std::map<std::tuple<int, Mono, Mono, Mono, Mono>, int> slot;
  std::vector<int> level;  // indexed by slot - acc_total (non-leaf slots), slot acc_total = zero
  std::vector<HrrInstr> instr;
  std::vector<int> instr_level;
  double flops = 0;

  int leaf(int ch, const Mono &e, const Mono &f) {
    const MonoSet &es = (*E)[ch], &fs = (*F)[ch];
    auto ie = es.idx.find(e), jf = fs.idx.find(f);
    if (ie == es.idx.end() || jf == fs.idx.end()) throw std::runtime_error("HRR leaf outside accumulator");
    return acc_off[ch] + ie->second * fs.size() + jf->second;
  }
  int lev(int s) const { return s < acc_total ? 0 : level[s - acc_total]; }
  int emit(HrrInstr in, int lv) {
    int s = acc_total + (int)level.size();
    if (s > 65000) throw std::runtime_error("HRR program too large");
    in.tgt = (uint16_t)s;
    level.push_back(lv);
    instr.push_back(in);
    instr_level.push_back(lv);
    return s;
  }
  int get(int ch, const Mono &a, const Mono &b, const Mono &c, const Mono &d) {
    if (mono_l(b) == 0 && mono_l(d) == 0) return leaf(ch, a, c);
    auto key = std::make_tuple(ch, a, b, c, d);
    auto it = slot.find(key);
    if (it != slot.end()) return it->second;
    HrrInstr in{};
    if (mono_l(d) > 0) {  // |c, d+1_i) = |c+1_i, d) + (C-D)_i |c, d)
      int i = first_dir(d);
      Mono d1 = shift(d, i, -1);
      in.kind = 1;
      in.dir = (uint8_t)i;
      in.s0 = (uint16_t)get(ch, a, b, shift(c, i, 1), d1);
      in.s1 = (uint16_t)get(ch, a, b, c, d1);
    } else {  // (a, b+1_i| = (a+1_i, b| + (A-B)_i (a, b|
      int i = first_dir(b);
      Mono b1 = shift(b, i, -1);
      in.kind = 0;
      in.dir = (uint8_t)i;
      in.s0 = (uint16_t)get(ch, shift(a, i, 1), b1, c, d);
      in.s1 = (uint16_t)get(ch, a, b1, c, d);
    }
    flops += 2;
    int s = emit(in, 1 + std::max(lev(in.s0), lev(in.s1)));
    slot[key] = s;
    return s;
  }
};

// Liveness-based slot assignment for a level-ordered program.  Entry k runs
// at level lev[k] (nondecreasing over the writers), writes node tgt[k] (or
// nothing when tgt[k] < 0) and reads the nodes in src[k]; nodes below `fixed`
// keep their numbers.  A node's slot returns to the free pool once every level
// that reads it has finished (the kernel synchronises the warp between levels,
// so a step of level L may take any slot whose last reader ran at a level < L);
// nodes marked in `pinned` are never released.  Returns the new number of every
// node and, in *size, the number of slots used (fixed ones included).
std::vector<int> assign_slots(int nnodes, int fixed, const std::vector<int> &lev,
                              const std::vector<int> &tgt, const std::vector<std::vector<int>> &src,
                              const std::vector<char> &pinned, int *size) {
  std::vector<int> last(nnodes, -1);
  for (size_t k = 0; k < tgt.size(); ++k)
    for (int x : src[k])
      if (x >= fixed) last[x] = std::max(last[x], lev[k]);
  std::vector<int> map(nnodes, -1);
  for (int x = 0; x < fixed; ++x) map[x] = x;
  std::set<int> pool;
  std::multimap<int, int> release;  // last-use level -> slot
  int next = fixed, cur = -1;
  for (size_t k = 0; k < tgt.size(); ++k) {
    if (tgt[k] < 0) continue;
    if (lev[k] < cur) throw std::runtime_error("assign_slots: writers out of level order");
    if (lev[k] != cur) {
      cur = lev[k];
      while (!release.empty() && release.begin()->first < cur) {
        pool.insert(release.begin()->second);
        release.erase(release.begin());
      }
    }
    int sl;
    if (!pool.empty()) {
      sl = *pool.begin();
      pool.erase(pool.begin());
    } else {
      sl = next++;
    }
    map[tgt[k]] = sl;
    if (!pinned[tgt[k]]) release.emplace(std::max(last[tgt[k]], lev[k]), sl);
  }
  *size = next;
  return map;
}

}  // namespace

void build_one_program(ProgramSet &ps, int la, int lb, int lc, int ld, int deriv, ClassProg &P) {
  P = ClassProg{};
  P.la = la; P.lb = lb; P.lc = lc; P.ld = ld;
  P.deriv = deriv;
  P.ltot = la + lb + lc + ld + (deriv ? 1 : 0);
  int lab = la + lb, lcd = lc + ld;
  // Accumulator channels: sets of bra monomials e and ket monomials f.
  std::vector<MonoSet> E, F;
  if (!deriv) {
    E.emplace_back(la, lab);
    F.emplace_back(lc, lcd);
  } else {
    // channel 0 (weight 1): lowered blocks (a-1 b|, (a b-1|, (ab|c-1 d);
    // a rectangle covering both of its needs.
    E.emplace_back(la - 1, lab);
    F.emplace_back(lc - 1, lcd);
    E.emplace_back(la + 1, lab + 1);  // channel 1 (2 alpha): (a+1 b|
    F.emplace_back(lc, lcd);
    E.emplace_back(la, lab + 1);      // channel 2 (2 beta): (a b+1|
    F.emplace_back(lc, lcd);
    E.emplace_back(la, lab);          // channel 3 (2 gamma): (ab|c+1 d)
    F.emplace_back(lc + 1, lcd + 1);
  }
  int nchan = (int)E.size();
  std::vector<int> acc_off(nchan + 1, 0);
  for (int c = 0; c < nchan; ++c) acc_off[c + 1] = acc_off[c] + E[c].size() * F[c].size();
  P.nchan = nchan;
  P.acc_total = acc_off[nchan];
  P.acc_size = P.acc_total;

  // VRR for every accumulator entry of every channel.
  VrrGen vg(P.ltot);
  std::vector<AccInstr> accs;
  for (int c = 0; c < nchan; ++c)
    for (int ie = 0; ie < E[c].size(); ++ie)
      for (int jf = 0; jf < F[c].size(); ++jf) {
        int s = vg.get(E[c].list[ie], F[c].list[jf], 0);
        AccInstr a{};
        a.slot = (uint16_t)s;
        a.acc = (uint16_t)(acc_off[c] + ie * F[c].size() + jf);
        a.chan = (uint8_t)c;
        accs.push_back(a);
      }
  // Level-sort VRR instructions (stable).
  {
    std::vector<int> order(vg.instr.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    // within a level, group steps by which optional terms they carry so that
    // the lanes of a warp mostly take the same branch
    auto type = [&](int k) { return (vg.instr[k].n1 ? 1 : 0) + (vg.instr[k].n2 ? 2 : 0); };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      if (vg.instr_level[x] != vg.instr_level[y]) return vg.instr_level[x] < vg.instr_level[y];
      return type(x) < type(y);
    });
    P.nh = 1;
    for (const VrrInstr &in : vg.instr) P.nh = std::max({P.nh, in.n1 + 1, in.n2 + 1});
    P.vrr_begin = (int)ps.vrr.size();
    P.vrr_level0 = (int)ps.levels.size();
    int cur = -1;
    for (int k : order) {
      if (vg.instr_level[k] != cur) {
        cur = vg.instr_level[k];
        ps.levels.push_back((int)ps.vrr.size());
      }
      ps.vrr.push_back(vg.instr[k]);
    }
    ps.levels.push_back((int)ps.vrr.size());
    P.nvrr_level = (int)ps.levels.size() - 1 - P.vrr_level0;
    P.vrr_flops = vg.flops;
    // compact the VRR region: slots of intermediates that no later level reads
    // are reused; the targets the accumulation reads stay to the end
    const int nnodes = (int)vg.level.size(), fixed = P.ltot + 2;
    std::vector<int> lev, tgt;
    std::vector<std::vector<int>> src;
    for (int k : order) {
      const VrrInstr &in = vg.instr[k];
      lev.push_back(vg.instr_level[k]);
      tgt.push_back(in.tgt);
      src.push_back({in.s0, in.s1, in.s2, in.s3, in.s4});
    }
    std::vector<char> pinned(nnodes, 0);
    for (const AccInstr &a : accs) pinned[a.slot] = 1;
    int size = 0;
    const std::vector<int> map = assign_slots(nnodes, fixed, lev, tgt, src, pinned, &size);
    for (int k = P.vrr_begin; k < (int)ps.vrr.size(); ++k) {
      VrrInstr &in = ps.vrr[k];
      in.tgt = (uint16_t)map[in.tgt];
      in.s0 = (uint16_t)map[in.s0];
      in.s1 = (uint16_t)map[in.s1];
      in.s2 = (uint16_t)map[in.s2];
      in.s3 = (uint16_t)map[in.s3];
      in.s4 = (uint16_t)map[in.s4];
    }
    for (AccInstr &a : accs) a.slot = (uint16_t)map[a.slot];
    P.vrr_size = size;
  }
  P.acc_begin = (int)ps.acc.size();
  P.nacc = (int)accs.size();
  ps.acc.insert(ps.acc.end(), accs.begin(), accs.end());

  // HRR to the outputs, in tiles.  Derivatives: nine tiles, one per (centre,
  // direction), each out[abcd] = chan_centre(raised) - n_x * chan0(lowered).
  // Plain integrals: tiles over ranges of a's Cartesian components, each the
  // row-major sub-block [a0, a0 + na) x [nb][nc][nd] of the output block; one
  // tile when the whole block's recurrence fits the slot budget, else the
  // fewest equal ranges that do (the output tiling of the paper's codegen
  // discussion; a tile recomputes the intermediates it shares with others).
  // Every tile reuses the same work region, so the region only has to hold
  // the largest tile.
  auto ma = monos(la), mb = monos(lb), mc = monos(lc), md = monos(ld);
  P.nout = ncart(la) * ncart(lb) * ncart(lc) * ncart(ld);
  const int blk = P.nout / ncart(la);  // outputs per a component
  struct Tile {
    TileProg T{};
    std::vector<HrrInstr> instr;   // level-ordered, slots final
    std::vector<int> bounds;       // level boundaries (indices into instr)
    double flops = 0;
  };
  // one tile: outputs with a in [a_lo, a_hi) (all for derivatives), for
  // derivative tile `dtile` (centre dtile / 3, direction dtile % 3) or -1
  auto make_tile = [&](int dtile, int a_lo, int a_hi) {
    Tile out;
    HrrGen hg;
    hg.E = &E;
    hg.F = &F;
    hg.acc_off = acc_off;
    hg.acc_total = P.acc_total;
    hg.level.push_back(0);  // slot acc_total: the zero slot
    const int zero = P.acc_total;
    std::vector<HrrInstr> final_instr;
    std::vector<int> final_level;
    const int centre = dtile / 3, x = dtile % 3;
    for (int ia = a_lo; ia < a_hi; ++ia) {
      const Mono &a = ma[ia];
      for (auto &b : mb)
        for (auto &c : mc)
          for (auto &d : md) {
            HrrInstr in{};
            in.kind = 2;  // t = s0 - n * s1
            if (dtile < 0) {
              int s = hg.get(0, a, b, c, d);
              in.s0 = (uint16_t)s;
              in.s1 = (uint16_t)zero;
              in.dir = 0;
              final_level.push_back(hg.lev(s) + 1);
            } else {
              int sr, sl = zero, n = 0;
              if (centre == 0) {
                sr = hg.get(1, shift(a, x, 1), b, c, d);
                if (a[x] > 0) { sl = hg.get(0, shift(a, x, -1), b, c, d); n = a[x]; }
              } else if (centre == 1) {
                sr = hg.get(2, a, shift(b, x, 1), c, d);
                if (b[x] > 0) { sl = hg.get(0, a, shift(b, x, -1), c, d); n = b[x]; }
              } else {
                sr = hg.get(3, a, b, shift(c, x, 1), d);
                if (c[x] > 0) { sl = hg.get(0, a, b, shift(c, x, -1), d); n = c[x]; }
              }
              in.s0 = (uint16_t)sr;
              in.s1 = (uint16_t)sl;
              in.dir = (uint8_t)n;
              final_level.push_back(1 + std::max(hg.lev(sr), hg.lev(sl)));
              hg.flops += 2;
            }
            final_instr.push_back(in);
          }
    }
    TileProg &T = out.T;
    T.nout = (int)final_instr.size();
    T.a0 = a_lo;
    T.na = a_hi - a_lo;
    T.store_off = (dtile < 0 ? 0 : dtile * P.nout) + a_lo * blk;
    const int nodes_end = hg.acc_total + (int)hg.level.size();  // first output node
    if (nodes_end + T.nout > 65000) throw std::runtime_error("HRR output block too large");
    for (size_t k = 0; k < final_instr.size(); ++k) {
      final_instr[k].tgt = (uint16_t)(nodes_end + k);
      hg.instr.push_back(final_instr[k]);
      hg.instr_level.push_back(final_level[k]);
    }
    std::vector<int> order(hg.instr.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int u, int v) { return hg.instr_level[u] < hg.instr_level[v]; });
    // Slots: accumulators and the zero slot keep their numbers, the output
    // block follows them contiguously, and the intermediates share a pool
    // above it by liveness.
    T.out_base = hg.acc_total + 1;
    const int fixed = hg.acc_total + 1;
    std::vector<int> lev, tgt;
    std::vector<std::vector<int>> src;
    for (int k : order) {
      const HrrInstr &in = hg.instr[k];
      lev.push_back(hg.instr_level[k]);
      tgt.push_back(in.tgt < nodes_end ? (int)in.tgt : -1);  // outputs are placed directly
      src.push_back({in.s0, in.s1});
    }
    int pool_size = 0;
    const std::vector<int> pool_map =
        assign_slots(nodes_end, fixed, lev, tgt, src, std::vector<char>(nodes_end, 0), &pool_size);
    const int pool_base = T.out_base + T.nout;
    auto remap = [&](int v) {
      if (v < fixed) return v;
      if (v >= nodes_end) return T.out_base + (v - nodes_end);
      return pool_base + (pool_map[v] - fixed);
    };
    int cur = -1;
    for (int k : order) {
      if (hg.instr_level[k] != cur) {
        cur = hg.instr_level[k];
        out.bounds.push_back((int)out.instr.size());
      }
      HrrInstr in = hg.instr[k];
      in.tgt = (uint16_t)remap(in.tgt);
      in.s0 = (uint16_t)remap(in.s0);
      in.s1 = (uint16_t)remap(in.s1);
      out.instr.push_back(in);
    }
    out.bounds.push_back((int)out.instr.size());
    T.nhrr_level = (int)out.bounds.size() - 1;
    T.hrr_size = 1 + T.nout + (pool_size - fixed);  // zero slot, outputs, pool
    if (P.acc_total + T.hrr_size > 65000) throw std::runtime_error("HRR tile too large");
    out.flops = hg.flops;
    return out;
  };
  // The fewest a-ranges whose tiles fit: plain integrals keep the class's
  // slots (accumulators and the larger of the vertical region and the tile's
  // horizontal region) within kTileSlotBudget, or, where the accumulators
  // and the vertical region alone exceed it, a horizontal region no larger
  // than the vertical one; every tile must fit the 16-bit slot indices (the
  // derivative tiles of the f classes split for that alone).  One component
  // per tile is the last resort.
  const int na = ncart(la);
  const int limit = deriv ? 1 << 30 : std::max(kTileSlotBudget, P.acc_total + P.vrr_size);
  auto ranged = [&](int dtile) {
    for (int nt = 1; nt <= na; ++nt) {
      const int chunk = (na + nt - 1) / nt;
      if (nt > 1 && (na + chunk - 1) / chunk != nt) continue;  // same ranges as a smaller count
      std::vector<Tile> cand;
      bool fits = true;
      try {
        for (int a0 = 0; a0 < na; a0 += chunk) {
          cand.push_back(make_tile(dtile, a0, std::min(na, a0 + chunk)));
          if (P.acc_total + std::max(P.vrr_size, cand.back().T.hrr_size) > limit) {
            fits = false;
            if (chunk > 1) break;  // try more tiles
          }
        }
      } catch (const std::runtime_error &) {
        if (chunk == 1) throw;
        fits = false;
      }
      if (fits || chunk == 1) return cand;
    }
    return std::vector<Tile>();
  };
  std::vector<Tile> tiles;
  if (deriv) {
    for (int t = 0; t < 9; ++t)
      for (Tile &x : ranged(t)) tiles.push_back(std::move(x));
  } else {
    tiles = ranged(-1);
  }
  P.ntile = (int)tiles.size();
  P.tile_begin = (int)ps.tiles.size();
  P.hrr_size = 0;
  P.hrr_flops = 0;
  for (Tile &t : tiles) {
    t.T.hrr_level0 = (int)ps.levels.size();
    const int base = (int)ps.hrr.size();
    for (size_t L = 0; L + 1 < t.bounds.size(); ++L) ps.levels.push_back(base + t.bounds[L]);
    ps.levels.push_back(base + t.bounds.back());
    ps.hrr.insert(ps.hrr.end(), t.instr.begin(), t.instr.end());
    P.hrr_size = std::max(P.hrr_size, t.T.hrr_size);
    P.hrr_flops += t.flops;
    ps.tiles.push_back(t.T);
  }
}

// Every slot a program touches must lie inside the regions the kernel sizes
// from the program's own counts; checked once, on the host, before any launch.
static void validate(const ProgramSet &ps, const ClassProg &P) {
  auto bad = [&](const char *what) {
    throw std::runtime_error(std::string("program (") + std::to_string(P.la) + std::to_string(P.lb) +
                             "|" + std::to_string(P.lc) + std::to_string(P.ld) + ") " + what);
  };
  const int v0 = ps.levels[P.vrr_level0], v1 = ps.levels[P.vrr_level0 + P.nvrr_level];
  for (int k = v0; k < v1; ++k) {
    const VrrInstr &in = ps.vrr[k];
    for (int sl : {(int)in.tgt, (int)in.s0, (int)in.s1, (int)in.s2, (int)in.s3, (int)in.s4})
      if (sl >= P.vrr_size) bad("VRR slot out of range");
    if (in.tgt <= P.ltot + 1) bad("VRR overwrites a base slot");
    if (in.kind > 1 || in.dir > 2) bad("VRR kind/dir");
    if (in.n1 >= kNhMax || in.n2 >= kNhMax || P.nh > kNhMax) bad("VRR multiplier");
  }
  // the steps of one level run concurrently on the lanes of a warp: none may
  // write a slot that the level reads, and no two may write the same slot
  auto level_hazards = [&](const std::vector<int> &reads, const std::vector<int> &writes) {
    std::set<int> w;
    for (int x : writes)
      if (!w.insert(x).second) bad("two steps of one level write the same slot");
    for (int x : reads)
      if (w.count(x)) bad("a level writes a slot that it reads");
  };
  for (int L = 0; L < P.nvrr_level; ++L) {
    std::vector<int> rd, wr;
    for (int k = ps.levels[P.vrr_level0 + L]; k < ps.levels[P.vrr_level0 + L + 1]; ++k) {
      const VrrInstr &in = ps.vrr[k];
      rd.insert(rd.end(), {in.s0, in.s1, in.s2, in.s3, in.s4});
      wr.push_back(in.tgt);
    }
    level_hazards(rd, wr);
  }
  for (int t = 0; t < P.ntile; ++t) {
    const TileProg &T = ps.tiles[P.tile_begin + t];
    for (int L = 0; L < T.nhrr_level; ++L) {
      std::vector<int> rd, wr;
      for (int k = ps.levels[T.hrr_level0 + L]; k < ps.levels[T.hrr_level0 + L + 1]; ++k) {
        rd.insert(rd.end(), {ps.hrr[k].s0, ps.hrr[k].s1});
        wr.push_back(ps.hrr[k].tgt);
      }
      level_hazards(rd, wr);
    }
  }
  for (int k = P.acc_begin; k < P.acc_begin + P.nacc; ++k) {
    const AccInstr &a = ps.acc[k];
    if (a.slot >= P.vrr_size || a.acc >= P.acc_total || a.chan >= P.nchan) bad("ACC index");
  }
  const int hmax = P.acc_total + P.hrr_size;
  for (int t = 0; t < P.ntile; ++t) {
    const TileProg &T = ps.tiles[P.tile_begin + t];
    const int h0 = ps.levels[T.hrr_level0], h1 = ps.levels[T.hrr_level0 + T.nhrr_level];
    for (int k = h0; k < h1; ++k) {
      const HrrInstr &in = ps.hrr[k];
      if (in.tgt >= hmax || in.s0 >= hmax || in.s1 >= hmax) bad("HRR slot out of range");
      if (in.tgt <= P.acc_total) bad("HRR overwrites an accumulator or the zero slot");
      if (in.kind > 2 || (in.kind < 2 && in.dir > 2)) bad("HRR kind/dir");
    }
    if (T.out_base + T.nout > hmax) bad("output block");
    const int blk = P.nout / ncart(P.la);
    if (T.na < 1 || T.a0 < 0 || T.a0 + T.na > ncart(P.la) || T.nout != T.na * blk) bad("tile range");
    const int comp = T.store_off / P.nout;  // derivative component (centre, direction); 0 for values
    if (T.store_off != comp * P.nout + T.a0 * blk || comp > (P.deriv ? 8 : 0)) bad("tile store offset");
  }
  {  // the tiles of each component cover the a components in order
    int comp = 0, next = 0;
    for (int t = 0; t < P.ntile; ++t) {
      const TileProg &T = ps.tiles[P.tile_begin + t];
      if (next == ncart(P.la)) {
        ++comp;
        next = 0;
      }
      if (T.store_off / P.nout != comp || T.a0 != next) bad("tiles out of order");
      next += T.na;
    }
    if (next != ncart(P.la) || comp != (P.deriv ? 8 : 0)) bad("tiles do not cover the block");
  }
}

void validate_program(const ProgramSet &ps, const ClassProg &P) { validate(ps, P); }

void build_programs(ProgramSet &ps) {
  ps = ProgramSet{};
  ps.progs.resize(2 * kNumPairClass * kNumPairClass);
  for (int deriv = 0; deriv <= 1; ++deriv)
    for (int la = 0; la <= (deriv ? kMaxLGrad : kMaxL); ++la)
      for (int lb = 0; lb <= la; ++lb)
        for (int lc = 0; lc <= (deriv ? kMaxLGrad : kMaxL); ++lc)
          for (int ld = 0; ld <= lc; ++ld)
            build_one_program(ps, la, lb, lc, ld, deriv, ps.progs[quartet_index(la, lb, lc, ld, deriv)]);
  for (const ClassProg &P : ps.progs)
    if (P.nout) validate(ps, P);  // derivative classes above kMaxLGrad stay empty
}

}  // namespace ltjk
