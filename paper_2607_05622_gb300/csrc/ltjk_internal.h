// Internal structures shared by the host code and the CUDA kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "ltjk.h"

namespace ltjk {

constexpr int kMaxL = LTJK_MAX_L;           // value build: s, p, d, f
constexpr int kMaxLGrad = LTJK_MAX_L_GRAD;  // gradient adjoint: s, p, d
constexpr int kMaxLDeriv = kMaxLGrad + 1;   // one raise for the derivative integrals
constexpr int kMaxPrim = 8;
constexpr int kMaxPrimPair = kMaxPrim * kMaxPrim;
// largest total angular momentum of a quartet program, value or derivative
constexpr int kMaxLtot = 4 * kMaxL > 4 * kMaxLGrad + 1 ? 4 * kMaxL : 4 * kMaxLGrad + 1;
constexpr int kBoysMaxM = kMaxLtot + 2;
// largest angular momentum on one side of a recurrence, and the integer
// multipliers n/2 a recurrence step takes (n up to that sum, plus one)
constexpr int kMaxSideL = 2 * kMaxL > 2 * kMaxLGrad + 1 ? 2 * kMaxL : 2 * kMaxLGrad + 1;
constexpr int kNhMax = kMaxSideL + 2;
// Slot budget of a value class's output tiling: accumulators plus the larger
// of the vertical region and one tile's horizontal region (8 bytes a slot in
// the FP64 classes: 16 KB).  On the 200-AO chain this tiles (dd|dd), (dd|dp)
// and (dp|dd) and measured 1.5 % faster than a budget that leaves every s/p/d
// class whole (8192); tiling every class whose horizontal region exceeds its
// vertical one (budget 0) measured 7 % slower (more HRR steps, fewer outputs
// per digestion pass).
constexpr int kTileSlotBudget = 2048;

#ifdef __CUDACC__
#define LTJK_HD __host__ __device__
#else
#define LTJK_HD
#endif

LTJK_HD constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// Coefficient slots of one primitive quartet, stored after its base values
// [00|00]^(m), m = 0..ltot, in the per-warp primitive table.
enum CoefSlot {
  kPAx = 0, kPAy, kPAz,   // bra step, first coefficient (P - A)
  kQCx, kQCy, kQCz,       // ket step, first coefficient (Q - C)
  kWPx, kWPy, kWPz,       // bra step, second coefficient (W - P)
  kWQx, kWQy, kWQz,       // ket step, second coefficient (W - Q)
  kHalfZeta,              // 1/(2 zeta)
  kHalfEta,               // 1/(2 eta)
  kRhoZeta,               // rho/zeta
  kRhoEta,                // rho/eta
  kHalfSum,               // 1/(2 (zeta+eta))
  kWA,                    // derivative channel weights: 2 alpha, 2 beta, 2 gamma
  kWB,
  kWC,
  kNumCoef
};

// One Obara-Saika step.  kind 0 (bra): raise e along dir
//   t = PA*s0 + WP*s1 + n1/(2zeta) (s2 - rho/zeta s3)
// kind 1 (ket): raise f along dir
//   t = QC*s0 + WQ*s1 + n1/(2eta) (s2 - rho/eta s3) + n2/(2(zeta+eta)) s4
struct VrrInstr {
  uint16_t tgt, s0, s1, s2, s3, s4;
  uint8_t kind, dir, n1, n2;
};
static_assert(sizeof(VrrInstr) == 16, "VrrInstr layout");

// One horizontal step t = s0 + X_dir * s1, X = A - B (kind 0) or C - D (kind 1).
struct HrrInstr {
  uint16_t tgt, s0, s1;
  uint8_t kind, dir;
};
static_assert(sizeof(HrrInstr) == 8, "HrrInstr layout");

// Accumulation of one VRR target into a contracted accumulator:
// acc[chan*acc_chan + acc] += weight(chan) * vrr[slot].
struct AccInstr {
  uint16_t slot, acc;
  uint8_t chan, pad0;
  uint16_t pad1;
};
static_assert(sizeof(AccInstr) == 8, "AccInstr layout");

// One output tile of a class program: HRR levels and the contiguous output block.
struct TileProg {
  int hrr_level0, nhrr_level;  // level ranges in ProgramSet::levels
  int out_base;                // HRR slot of output 0 (outputs contiguous)
  int nout;                    // outputs of the tile (na nb nc nd, na = this tile's a range)
  int hrr_size;                // HRR slots beyond the accumulators this tile uses
  int a0, na;                  // a's Cartesian components [a0, a0 + na) (derivatives: all)
  int store_off;               // offset of the tile's first output in the stored blocks:
                               // value a0 nb nc nd; derivative tile * (na nb nc nd)
};

// Device view of one class program (offsets into the shared instruction pools).
struct ClassProg {
  int la, lb, lc, ld, ltot;  // ltot includes the derivative raise when deriv
  int deriv;                 // 0: plain integrals; 1: derivative channels
  int nchan;                 // accumulator channels (1 plain, 4 deriv)
  int vrr_begin, nvrr_level;  // level ranges are in level_pool[vrr_level0 .. +nvrr_level]
  int vrr_level0;
  int acc_begin, nacc;
  int ntile, tile_begin;     // output tiles (plain: ranges of a; 9 = centre A,B,C x xyz for deriv)
  int vrr_size;   // slots of one VRR region (slot 0 = zero, 1..ltot+1 = base values)
  int acc_size;   // slots of one accumulator channel
  int hrr_size;   // HRR slots beyond the accumulators, max over tiles (slot acc_total = zero)
  int acc_total;  // nchan * acc_size
  int nout;       // outputs of the whole block (na nb nc nd); derivatives: per tile
  int nh;         // 1 + largest integer multiplier of a VRR step
  double vrr_flops, hrr_flops;  // flop model: per primitive quartet / per contracted quartet
};

struct ProgramSet {
  std::vector<VrrInstr> vrr;
  std::vector<HrrInstr> hrr;
  std::vector<AccInstr> acc;
  std::vector<int> levels;        // level boundaries (instruction index), per program
  std::vector<TileProg> tiles;
  std::vector<ClassProg> progs;   // index = class_index(la,lb,lc,ld,deriv)
};

// Class index of (la,lb,lc,ld) with la>=lb, lc>=ld (any bra/ket order).
inline int pair_class(int la, int lb) { return la * (la + 1) / 2 + lb; }
constexpr int kNumPairClass = (kMaxL + 1) * (kMaxL + 2) / 2;
inline int quartet_index(int la, int lb, int lc, int ld, int deriv) {
  return (deriv * kNumPairClass + pair_class(la, lb)) * kNumPairClass + pair_class(lc, ld);
}

// Value classes whose J/K digestion runs in the class-specialised kernel: one
// thread evaluates a whole contracted quartet, so only classes whose
// straight-line code fits 128 registers (four warps of 128 threads per SM
// scheduler group) with at most a few hundred bytes of spills are listed:
// total angular momentum up to 3 with everything in registers, and the
// classes of total angular momentum 4 with at most 54 integrals ((dd|ss),
// (ds|ds), (dp|ps), (ds|pp)) with their contracted accumulators and output
// block in shared memory.  (pp|pp) and heavier classes spill kilobytes per
// thread and run in the warp-cooperative interpreted kernel.
LTJK_HD constexpr bool gen_class(int la, int lb, int lc, int ld) {
  return la >= lb && lc >= ld && (la > lc || (la == lc && lb >= ld)) &&
         (la + lb + lc + ld <= 3 || (la + lb + lc + ld == 4 && ncart(la) * ncart(lb) * ncart(lc) * ncart(ld) <= 54));
}

// Classes whose FP64-class quartets run in IEEE binary64 instead of
// double-float: those with an f shell.  Their vertical and horizontal
// recurrences amplify rounding about 1e4-fold relative to Q_ab Q_cd (f
// shells next to d shells of exponent ~1e3), which at double-float's
// ~2^-44 per operation reached 1.7e-10 of max|K| on a 200-AO f-shell chain,
// above the FP64 gate; binary64 leaves 4e-13.  s/p/d classes amplify less and
// stay double-float.
LTJK_HD constexpr bool ieee64_class(int la, int lb, int lc, int ld) {
  return la >= 3 || lb >= 3 || lc >= 3 || ld >= 3;
}

void build_programs(ProgramSet &ps);
void build_one_program(ProgramSet &ps, int la, int lb, int lc, int ld, int deriv, ClassProg &out);
// The checks build_programs applies to every program (slots in range, no
// level writing a slot it reads, tiles covering the block), for a program
// built on its own; throws std::runtime_error.
void validate_program(const ProgramSet &ps, const ClassProg &P);
// Straight-line C++/CUDA source of one class program (codegen.cpp).
std::string emit_class_source(const ProgramSet &ps, int la, int lb, int lc, int ld, int deriv,
                              const std::string &prefix);

}  // namespace ltjk
