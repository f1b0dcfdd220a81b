// Straight-line source for one class program.
//
// The integral kernel interprets each class's recurrence program from shared
// memory: every step decodes an instruction and reads and writes numbered
// slots.  This generator turns the same program into straight-line C++/CUDA:
// every Obara-Saika step becomes one expression over named temporaries (the
// compiler keeps them in registers), every accumulation a fused multiply-add
// into the contracted accumulators, every horizontal step one expression, in
// the same operation order as the kernel's steps (product, then fused
// multiply-adds).  Terms that read the zero slot are dropped.  The emitted
// functions are templates over the arithmetic type, marked for host and
// device, so the same text is checked on the CPU and compiled for the GPU.
//
// Output, for a class (la lb|lc ld) with deriv 0/1 and a name prefix P:
//   template <typename Real, int AS = 1> LTJK_GEN_FN void P_vrr(const Real *base,
//       const Real *cf, const Real *h, Real *acc);
//     one primitive quartet: base[m] = [00|00]^(m), m = 0..ltot; cf the
//     kNumCoef coefficients of CoefSlot; h the 3 nh tables n/(2 zeta),
//     n/(2 eta), n/(2 (zeta+eta)); accumulator i, acc[AS * i], accumulated in
//     place (AS > 1: one column of a lane-interleaved shared-memory block).
//   template <typename Real, int AS = 1, int OS = 1> LTJK_GEN_FN void P_hrr(
//       const Real *acc, const Real *X, Real *out);
//     contracted accumulators acc[AS * i] -> output tiles out[OS * (store_off
//     + o)] (the tile's place in the block, or tile * nout for derivative
//     tiles); X[0..2] = A - B, X[3..5] = C - D.
// LTJK_GEN_FN is the function qualifier, defined by whoever includes the
// emitted text (inline host+device code for the CPU checks, forced-inline
// device code in the library).
#include <map>
#include <sstream>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "ltjk_internal.h"

namespace ltjk {

namespace {

// Operand of an expression: empty for an exact zero.
struct Val {
  std::string expr;
  bool zero() const { return expr.empty(); }
};

// a*b + c in the kernel's order: a product first, then fused multiply-adds.
std::string fma_chain(const std::vector<std::pair<std::string, std::string>> &terms) {
  std::string e;
  for (const auto &t : terms) {
    if (e.empty())
      e = t.first + " * " + t.second;
    else
      e = "fma(" + t.first + ", " + t.second + ", " + e + ")";
  }
  return e;
}

}  // namespace

std::string emit_class_source(const ProgramSet &ps, int la, int lb, int lc, int ld, int deriv,
                              const std::string &prefix) {
  if (la < lb || lc < ld || la > kMaxL || lc > kMaxL || lb < 0 || ld < 0 || (deriv != 0 && deriv != 1))
    throw std::invalid_argument("emit_class_source: class outside the program set");
  const ClassProg &p = ps.progs[quartet_index(la, lb, lc, ld, deriv)];
  std::ostringstream o;
  o << "// (" << la << lb << "|" << lc << ld << ")" << (deriv ? " derivative" : "")
    << " class: " << (ps.levels[p.vrr_level0 + p.nvrr_level] - ps.levels[p.vrr_level0])
    << " vertical steps, " << p.nacc << " accumulations, " << p.ntile << " output tile(s) of "
    << p.nout << "\n";

  // ---- vertical recurrence and accumulation, one primitive quartet
  o << "template <typename Real, int AS = 1>\nLTJK_GEN_FN void " << prefix
    << "_vrr(const Real *__restrict__ base, const Real *__restrict__ cf, const Real *__restrict__ h,\n"
    << "    Real *__restrict__ acc) {\n";
  o << "#ifndef __CUDA_ARCH__\n  using std::fma;\n#endif\n";
  std::map<int, Val> slot;  // slot -> current value
  for (int m = 0; m <= p.ltot; ++m) slot[1 + m] = Val{"base[" + std::to_string(m) + "]"};
  auto get = [&](int s) -> Val {
    if (s == 0) return Val{};
    auto it = slot.find(s);
    if (it == slot.end()) throw std::runtime_error("emit_class_source: VRR slot read before written");
    return it->second;
  };
  auto cf = [](int k) { return std::string("cf[") + std::to_string(k) + "]"; };
  int nv = 0;
  for (int L = 0; L < p.nvrr_level; ++L) {
    // a level never writes a slot it reads: read all sources of the level
    // before publishing its targets
    std::vector<std::pair<int, Val>> writes;
    for (int k = ps.levels[p.vrr_level0 + L]; k < ps.levels[p.vrr_level0 + L + 1]; ++k) {
      const VrrInstr &in = ps.vrr[k];
      std::vector<std::pair<std::string, std::string>> terms;
      const Val s0 = get(in.s0), s1 = get(in.s1);
      if (!s0.zero()) terms.push_back({cf(kPAx + 3 * in.kind + in.dir), s0.expr});
      if (!s1.zero()) terms.push_back({cf(kWPx + 3 * in.kind + in.dir), s1.expr});
      if (in.n1) {
        const Val s2 = get(in.s2), s3 = get(in.s3);
        const std::string hn = "h[" + std::to_string(in.kind * p.nh + in.n1) + "]";
        std::string inner;
        if (!s3.zero())
          inner = s2.zero() ? "(-" + cf(kRhoZeta + in.kind) + " * " + s3.expr + ")"
                            : "fma(-" + cf(kRhoZeta + in.kind) + ", " + s3.expr + ", " + s2.expr + ")";
        else if (!s2.zero())
          inner = s2.expr;
        if (!inner.empty()) terms.push_back({hn, inner});
      }
      if (in.n2) {
        const Val s4 = get(in.s4);
        if (!s4.zero()) terms.push_back({"h[" + std::to_string(2 * p.nh + in.n2) + "]", s4.expr});
      }
      if (terms.empty()) {
        writes.push_back({in.tgt, Val{}});
        continue;
      }
      const std::string name = "v" + std::to_string(nv++);
      o << "  const Real " << name << " = " << fma_chain(terms) << ";\n";
      writes.push_back({in.tgt, Val{name}});
    }
    for (auto &w : writes) slot[w.first] = w.second;
  }
  for (int k = p.acc_begin; k < p.acc_begin + p.nacc; ++k) {
    const AccInstr &in = ps.acc[k];
    const Val v = get(in.slot);
    if (v.zero()) continue;
    const std::string a = "acc[AS * " + std::to_string(in.acc) + "]";
    if (in.chan == 0)
      o << "  " << a << " += " << v.expr << ";\n";
    else
      o << "  " << a << " = fma(" << cf(kWA + in.chan - 1) << ", " << v.expr << ", " << a << ");\n";
  }
  o << "}\n\n";

  // ---- horizontal recurrence on the contracted accumulators, every tile
  o << "template <typename Real, int AS = 1, int OS = 1>\nLTJK_GEN_FN void " << prefix
    << "_hrr(const Real *__restrict__ acc, const Real *__restrict__ X, Real *__restrict__ out) {\n";
  o << "#ifndef __CUDA_ARCH__\n  using std::fma;\n#endif\n";
  for (int tile = 0; tile < p.ntile; ++tile) {
    const TileProg &T = ps.tiles[p.tile_begin + tile];
    std::map<int, Val> hs;
    auto hget = [&](int s) -> Val {
      auto it = hs.find(s);
      if (it != hs.end()) return it->second;
      if (s < p.acc_total) return Val{"acc[AS * " + std::to_string(s) + "]"};
      if (s == p.acc_total) return Val{};
      throw std::runtime_error("emit_class_source: HRR slot read before written");
    };
    int nh = 0;
    o << "  {  // tile " << tile << "\n";
    for (int L = 0; L < T.nhrr_level; ++L) {
      std::vector<std::pair<int, Val>> writes;
      for (int k = ps.levels[T.hrr_level0 + L]; k < ps.levels[T.hrr_level0 + L + 1]; ++k) {
        const HrrInstr &in = ps.hrr[k];
        const Val s0 = hget(in.s0), s1 = hget(in.s1);
        std::string c;
        if (in.kind < 2)
          c = "X[" + std::to_string(3 * in.kind + in.dir) + "]";
        else if (in.dir != 0)
          c = "Real(" + std::to_string(-(int)in.dir) + ")";
        std::string e;
        if (!c.empty() && !s1.zero())
          e = s0.zero() ? c + " * " + s1.expr : "fma(" + c + ", " + s1.expr + ", " + s0.expr + ")";
        else if (!s0.zero())
          e = s0.expr;
        if (e.empty()) {
          writes.push_back({in.tgt, Val{}});
          continue;
        }
        const std::string name = "t" + std::to_string(nh++);
        o << "    const Real " << name << " = " << e << ";\n";
        writes.push_back({in.tgt, Val{name}});
      }
      for (auto &w : writes) hs[w.first] = w.second;
    }
    for (int q = 0; q < T.nout; ++q) {
      const Val v = hget(T.out_base + q);
      o << "    out[OS * " << T.store_off + q << "] = " << (v.zero() ? "Real(0)" : v.expr) << ";\n";
    }
    o << "  }\n";
  }
  o << "}\n";
  return o.str();
}

}  // namespace ltjk
