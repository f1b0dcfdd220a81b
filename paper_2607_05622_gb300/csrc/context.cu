// C-ABI entry points of the library (include/ltjk.h): contexts, shell pairs and
// Schwarz screening, work lists, the J/K build, the gradient adjoint, the
// pseudo-densities and the inspection call.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "gen_kernel.cuh"
#include "host.h"
#include "kernels.cuh"

using namespace ltjk;

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_error(LTJK_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));      \
  } while (0)

namespace {

std::atomic<unsigned long long> g_launches{0};  // kernels launched by this library

constexpr int kKetChunk = 1;  // ket pairs per work item of the interpreted kernel: one quartet per
                              // warp balances best (16 per item measured 4-5 % slower)
constexpr int kGenKetChunk = 32;         // most ket pairs per work item (class-specialised kernel)
constexpr long long kTargetItems = 152 * 24;  // work items a class should offer the GPU
constexpr int kSideStreams = 4;          // class launches of one build run on these concurrently
constexpr int kSmemBudget = 200 * 1024;  // bytes of shared memory per CTA we plan for
constexpr int kMaxSmem = 227 * 1024;
constexpr int kSmemPerSM = 228 * 1024;      // shared memory of one SM
constexpr int kSmemPerCTAReserved = 1024;   // the driver's share of each CTA
constexpr int kRegsPerSM = 65536;
constexpr int kMaxCTAsPerSM = 32;
constexpr double kPrimPairDrop = 1e-18;  // drop primitive pair iff K_AB |c_a c_b| below this

// Device buffer owned by a context.  Stream-ordered allocation
// (cudaMallocAsync / cudaFreeAsync on the given stream, default: the legacy
// stream) never synchronises the whole device, so contexts can be created and
// destroyed while other work (another request, the service) runs.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, 0);
  }
  int alloc(size_t n, cudaStream_t st = 0) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
    if (n == 0) return LTJK_OK;
    cudaError_t e = cudaMallocAsync(&p, n, st);
    if (e != cudaSuccess) {
      p = nullptr;
      return set_error(LTJK_ENOMEM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
    }
    bytes = n;
    return LTJK_OK;
  }
  template <typename T>
  int upload(const std::vector<T> &v) {
    int rc = alloc(v.size() * sizeof(T));
    if (rc) return rc;
    if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return LTJK_OK;
  }
  template <typename T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

struct ClassWork {
  int X, Y;            // bra and ket pair class
  int la, lb, lc, ld;
  int ket_base;        // first pair of class Y in the sorted pair array
  DevBuf items64, items32;
  int n64 = 0, n32 = 0;
};

// Double-float pair (hi, lo) of a double: hi = nearest float, lo = nearest
// float to the remainder.
float2 split2(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// Streaming multiprocessors of the current device (grid sizing).
int num_sms() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  cache[dev] = n;
  return n;
}

// Programs are generated once per process and uploaded once per device.
struct ProgramCache {
  std::mutex mu;
  bool built = false;
  ProgramSet ps;
  std::map<int, std::shared_ptr<DevBuf>> vrr, hrr, acc, lev, tiles, boys, boys2;
};
ProgramCache g_prog;

int program_set(const ProgramSet **ps) {
  std::lock_guard<std::mutex> g(g_prog.mu);
  if (!g_prog.built) {
    try {
      build_programs(g_prog.ps);
    } catch (const std::exception &e) {
      return set_error(LTJK_EINVAL, "program generation failed: %s", e.what());
    }
    g_prog.built = true;
  }
  *ps = &g_prog.ps;
  return LTJK_OK;
}

int device_programs(int dev, DevProgs *out, const double **boys, const float2 **boys2) {
  const ProgramSet *ps;
  int rc = program_set(&ps);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(g_prog.mu);
  if (!g_prog.vrr.count(dev)) {
    auto v = std::make_shared<DevBuf>(), h = std::make_shared<DevBuf>(),
         a = std::make_shared<DevBuf>(), l = std::make_shared<DevBuf>(),
         t = std::make_shared<DevBuf>(), b = std::make_shared<DevBuf>();
    if ((rc = v->upload(ps->vrr)) || (rc = h->upload(ps->hrr)) || (rc = a->upload(ps->acc)) ||
        (rc = l->upload(ps->levels)) || (rc = t->upload(ps->tiles)))
      return rc;
    // tab[k][m][j] = F_{m+j}(T_k) / j!
    std::vector<double> raw((size_t)kBoysRows * kBoysRaw);
    boys_table(kBoysRows, kBoysRaw, kBoysStep, raw.data());
    std::vector<double> tab((size_t)kBoysRows * kBoysM * kBoysTaylor);
    for (int k = 0; k < kBoysRows; ++k)
      for (int m = 0; m < kBoysM; ++m) {
        double fact = 1.0;
        for (int j = 0; j < kBoysTaylor; ++j) {
          if (j > 0) fact *= j;
          tab[((size_t)k * kBoysM + m) * kBoysTaylor + j] = raw[(size_t)k * kBoysRaw + m + j] / fact;
        }
      }
    if ((rc = b->upload(tab))) return rc;
    // double-float table: row k (T_k = k/16) holds F_{m+j}(T_k)/j! for
    // m = 0..kBoysMaxM, then e^{-T_k}/j!, j < kBoysDfTaylor
    const int nraw = kBoysDfOrders + kBoysDfTaylor - 1;
    std::vector<double> raw2((size_t)kBoysDfRows * nraw);
    boys_table(kBoysDfRows, nraw, 1.0 / 16, raw2.data());
    std::vector<float2> tab2((size_t)kBoysDfRows * kBoysDfRow);
    for (int k = 0; k < kBoysDfRows; ++k) {
      double fact = 1.0;
      for (int j = 0; j < kBoysDfTaylor; ++j) {
        if (j > 0) fact *= j;
        for (int m = 0; m < kBoysDfOrders; ++m)
          tab2[(size_t)k * kBoysDfRow + m * kBoysDfTaylor + j] = split2(raw2[(size_t)k * nraw + m + j] / fact);
        tab2[(size_t)k * kBoysDfRow + kBoysDfOrders * kBoysDfTaylor + j] = split2(std::exp(-k / 16.0) / fact);
      }
    }
    auto b2 = std::make_shared<DevBuf>();
    if ((rc = b2->upload(tab2))) return rc;
    g_prog.boys2[dev] = b2;
    double inv_odd[kBoysRaw + 2], half_n[kNhMax];
    for (int m = 0; m < kBoysRaw + 2; ++m) inv_odd[m] = 1.0 / (2 * m + 1);
    for (int n = 0; n < kNhMax; ++n) half_n[n] = 0.5 * n;
    CUDA_TRY(cudaMemcpyToSymbol(c_inv_odd, inv_odd, sizeof(inv_odd)));
    CUDA_TRY(cudaMemcpyToSymbol(c_half_n, half_n, sizeof(half_n)));
    g_prog.vrr[dev] = v;
    g_prog.hrr[dev] = h;
    g_prog.acc[dev] = a;
    g_prog.lev[dev] = l;
    g_prog.tiles[dev] = t;
    g_prog.boys[dev] = b;
  }
  out->vrr = g_prog.vrr[dev]->as<VrrInstr>();
  out->hrr = g_prog.hrr[dev]->as<HrrInstr>();
  out->acc = g_prog.acc[dev]->as<AccInstr>();
  out->levels = g_prog.lev[dev]->as<int>();
  out->tiles = g_prog.tiles[dev]->as<TileProg>();
  *boys = g_prog.boys[dev]->as<double>();
  *boys2 = g_prog.boys2[dev]->as<float2>();
  return LTJK_OK;
}

// Launch configuration of one class program: groups per warp from the average
// width of a recurrence level, warps per CTA from the shared-memory budget.
ClassLaunch make_launch(const ClassProg &p, size_t real_bytes) {
  // Candidate layouts: G groups of S lanes, each group running P = 2 or 1
  // primitive quartets (its S lanes over the independent steps of each
  // recurrence level), and a T-entry primitive table (PG <= T; T shrinks
  // from 32 while the warp's shared memory would keep fewer than 16 warps on
  // an SM, as long as the digestion's offset table still fits in it).  Cost
  // per primitive quartet, in warp iterations: sum over levels of
  // ceil(width / S) x S / 64 for P = 2 (one step per lane per iteration,
  // applied to two quartets) or ceil(width / 2S) x S / 32 for P = 1 (two
  // steps of one quartet per lane per iteration), scaled by
  // 16 / (warps per SM) when shared memory allows fewer than 16 warps (a
  // target of 12 measured 1 % slower, 8 measured 13 % slower).  The
  // cheapest layout wins; narrow levels favour small S, large programs
  // large S (their slots are G-fold).
  const ProgramSet &ps = g_prog.ps;
  ClassLaunch best{};
  double best_cost = 1e300;
  for (int P = 2; P >= 1; --P)
  for (int S = 32; S >= 1; S /= 2) {
    if (P * (32 / S) > 32) continue;  // the table holds 32 entries: PG of them in flight
    ClassLaunch cl{};
    cl.p = p;
    cl.G = 32 / S;
    cl.P = P;
    cl.T = 32;
    cl.smem_per_warp = (int)warp_smem_bytes(p, cl.G, cl.T, P, real_bytes);
    while (cl.T > 8 && cl.T / 2 >= P * cl.G && cl.smem_per_warp > kSmemPerSM / 16 &&
           (size_t)(cl.T / 2) * pt_stride(p) * real_bytes >= digest_table_bytes(p)) {
      cl.T /= 2;
      cl.smem_per_warp = (int)warp_smem_bytes(p, cl.G, cl.T, P, real_bytes);
    }
    if (cl.smem_per_warp > kSmemBudget) continue;
    double cost = 0.0;
    for (int L = 0; L < p.nvrr_level; ++L) {
      const int w = ps.levels[p.vrr_level0 + L + 1] - ps.levels[p.vrr_level0 + L];
      cost += P == 2 ? (double)((w + S - 1) / S) * S / 64.0 : (double)((w + 2 * S - 1) / (2 * S)) * S / 32.0;
    }
    cost += 1.0 / 32.0;  // per-quartet overheads: set-up share, syncs
    // P = 1 loads each step's instruction for one quartet only: weighted by
    // 1.25 (the factor that measured best; 1 gave 3 % fewer gradients/s,
    // 1.5 and 1.75 3-5 % slower f-shell builds; P = 4 measured 2 % slower)
    if (P == 1) cost *= 1.25;
    const int warps_sm = std::min(16, kSmemPerSM / (cl.smem_per_warp + kSmemPerCTAReserved));
    if (warps_sm < 16) cost *= 16.0 / std::max(warps_sm, 1);
    if (cost < best_cost * 0.98) {  // a smaller S must win by 2 %: larger S needs less shared memory
      best_cost = cost;
      best = cl;
    }
  }
  if (best_cost == 1e300) {  // nothing within the budget: one group, smallest table
    best.p = p;
    best.G = 1;
    best.T = 8;
    best.P = 1;
    best.smem_per_warp = (int)warp_smem_bytes(p, 1, 8, 1, real_bytes);
  }
  best.warps = std::max(1, std::min(4, kSmemBudget / std::max(best.smem_per_warp, 1)));
  best.split = 1;
  return best;
}

// Layout of a derivative class in the gradient: as make_launch, and for the
// classes whose J/K build is class-specialised (work items of up to
// kGenKetChunk kets, one per lane there) one warp per ket of an item.
ClassLaunch grad_launch(const ClassProg &p, size_t real_bytes) {
  ClassLaunch cl = make_launch(p, real_bytes);
  if (gen_class(p.la, p.lb, p.lc, p.ld)) cl.split = kGenKetChunk;
  return cl;
}

// Warps per CTA that put the most warps on an SM, given the shared memory one
// warp needs and the kernel's registers per thread: a heavy class whose warp
// needs 30 KB fits seven one-warp CTAs on an SM but only one four-warp CTA.
int warps_per_cta(int smem_per_warp, int regs) {
  const int regs_per_warp = ((regs + 7) / 8 * 8) * 32;
  int best_w = 1, best = 0;
  for (int w : {4, 2, 1}) {
    if (w > 1 && w * smem_per_warp > kSmemBudget) continue;
    const int by_smem = kSmemPerSM / (w * smem_per_warp + kSmemPerCTAReserved);
    const int by_regs = kRegsPerSM / (regs_per_warp * w);
    const int ctas = std::min({by_smem, by_regs, kMaxCTAsPerSM});
    if (ctas * w > best) {
      best = ctas * w;
      best_w = w;
    }
  }
  return best_w;
}

template <typename Real, int MODE>
int launch_class(const DevProgs &PR, const ClassLaunch &cl_in, const JobTable &T, cudaStream_t st) {
  if (T.total <= 0) return LTJK_OK;
  static std::atomic<int> regs{0};  // per instantiation
  if (regs.load() == 0) {
    CUDA_TRY(cudaFuncSetAttribute(quartet_kernel<Real, MODE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    cudaFuncAttributes fa{};
    CUDA_TRY(cudaFuncGetAttributes(&fa, quartet_kernel<Real, MODE>));
    regs.store(fa.numRegs > 0 ? fa.numRegs : 128);
  }
  ClassLaunch cl = cl_in;
  cl.split = std::max(cl.split, 1);
  cl.warps = warps_per_cta(cl.smem_per_warp, regs.load());
  const size_t smem = (size_t)cl.smem_per_warp * cl.warps;
  if (smem > (size_t)kMaxSmem)
    return set_error(LTJK_EUNSUPPORTED, "class (%d%d|%d%d) needs %zu bytes of shared memory",
                     cl.p.la, cl.p.lb, cl.p.lc, cl.p.ld, smem);
  const long long units = (long long)T.total * std::max(cl.split, 1);
  const int grid = (int)((units + cl.warps - 1) / cl.warps);  // one warp per unit, not persistent
  quartet_kernel<Real, MODE><<<grid, 32 * cl.warps, smem, st>>>(PR, cl, T);
  CUDA_TRY(cudaGetLastError());
  g_launches += 1;
  return LTJK_OK;
}

// Class-specialised J/K kernel of class (LA LB|LC LD): four warps per CTA, a
// CTA per four work items.
template <typename Real, int LA, int LB, int LC, int LD>
int launch_gen_cls(const JobTable &T, cudaStream_t st) {
  if (T.total <= 0) return LTJK_OK;
  constexpr int NOUT = ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD);
  constexpr int NACC = kGenSmemAcc<LA, LB, LC, LD> ? GenClass<LA, LB, LC, LD>::kAcc : 0;
  constexpr int kWarps = 4;
  const size_t smem = gen_warp_smem<NOUT, NACC, Real>() * kWarps;
  static std::atomic<int> configured{0};  // per instantiation
  auto kern = gen_jk_kernel<Real, LA, LB, LC, LD>;
  if (configured.load() == 0) {
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured.store(1);
  }
  // one warp per work item, no persistent CTAs: each CTA retires after its
  // items, so SMs turn over every few hundred microseconds and concurrent
  // launches (other classes, higher-priority streams of the service) get
  // them without waiting for this launch to end
  const int grid = (T.total + kWarps - 1) / kWarps;
  kern<<<grid, 32 * kWarps, smem, st>>>(T);
  CUDA_TRY(cudaGetLastError());
  g_launches += 1;
  return LTJK_OK;
}

template <typename Real>
int launch_gen(int la, int lb, int lc, int ld, const JobTable &T, cudaStream_t st) {
#define LTJK_GEN_CASE(A_, B_, C_, D_) \
  if (la == A_ && lb == B_ && lc == C_ && ld == D_) return launch_gen_cls<Real, A_, B_, C_, D_>(T, st);
  LTJK_GEN_CLASSES(LTJK_GEN_CASE)
#undef LTJK_GEN_CASE
  return set_error(LTJK_EINVAL, "no class-specialised kernel for (%d%d|%d%d)", la, lb, lc, ld);
}

// J/K launch of one class: the class-specialised kernel where the class has
// one, the interpreted kernel otherwise.
template <typename Real>
int launch_jk(const ClassProg &p, const DevProgs &PR, const JobTable &T, cudaStream_t st) {
  if (gen_class(p.la, p.lb, p.lc, p.ld)) return launch_gen<Real>(p.la, p.lb, p.lc, p.ld, T, st);
  return launch_class<Real, kJK>(PR, make_launch(p, sizeof(Real)), T, st);
}

// A launch over one job.
JobTable single_job(const DevBasis &B, const JKArgs &a, const WorkItem *items, int n) {
  JobTable T;
  T.njobs = 1;
  T.total = n;
  T.j[0].B = B;
  T.j[0].a = a;
  T.j[0].items = items;
  T.j[0].nitems = n;
  T.j[0].first = 0;
  return T;
}

}  // namespace

// ------------------------------------------------------------------ context
struct ltjk_ctx {
  int device = 0;
  ltjk_opts opts{};
  int natoms = 0, nshells = 0, nao = 0, npairs = 0;
  // binary64 copies of the densities beside the double-float ones: a context
  // with an f shell in an FP64-class or mixed mode runs those classes in
  // IEEE binary64 (ieee64_class), whose digestion reads binary64 densities
  bool ieee_copies = false;
  std::vector<double> coords;
  std::vector<int> sh_l, sh_atom, sh_ao, sh_nprim, sh_p0;
  std::vector<double> exps, ncoef;
  // sorted pairs
  std::vector<int2> pair_sh;
  std::vector<double> pair_Q;
  std::vector<int> class_begin;  // pair index range of each pair class
  std::map<std::pair<int, int>, int> pair_of;  // canonical (a,b) -> sorted pair index
  // device data
  DevBuf d_ctr, d_l, d_ao, d_atom, d_pair_sh, d_pair_pp0, d_pair_npp, d_pp_zeta, d_pp_izeta, d_pp_P,
      d_pp_pref, d_pp_a, d_pp_b, d_pp2, d_ctr2, d_ppg2, d_ppg;
  DevProgs progs{};
  const double *boys = nullptr;
  const float2 *boys2 = nullptr;
  std::vector<std::unique_ptr<ClassWork>> work;       // value build
  DevBuf scratch;
  DevBuf d_sph;   // Cartesian -> real-spherical matrix T [nsph][nao], built on first use
  int nsph = 0;
  DevBuf d_t;
  ltjk_ctx_stats stats{};
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSideStreams] = {};
  ~ltjk_ctx() {
    for (int k = 0; k < kSideStreams; ++k) {
      if (side[k]) cudaStreamDestroy(side[k]);
      if (join_ev[k]) cudaEventDestroy(join_ev[k]);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
  }

  DevBasis basis() const {
    DevBasis B{};
    B.sh_ctr = d_ctr.as<double>();
    B.sh_l = d_l.as<int>();
    B.sh_ao = d_ao.as<int>();
    B.sh_atom = d_atom.as<int>();
    B.pair_sh = d_pair_sh.as<int2>();
    B.pair_pp0 = d_pair_pp0.as<int>();
    B.pair_npp = d_pair_npp.as<int>();
    B.pp_zeta = d_pp_zeta.as<double>();
    B.pp_inv_zeta = d_pp_izeta.as<double>();
    B.pp_P = d_pp_P.as<double>();
    B.pp_pref = d_pp_pref.as<double>();
    B.pp_a = d_pp_a.as<double>();
    B.pp_b = d_pp_b.as<double>();
    B.pp2 = d_pp2.as<float2>();
    B.ctr2 = d_ctr2.as<float2>();
    B.boys = boys;
    B.ppg2 = d_ppg2.as<float2>();
    B.ppg = d_ppg.as<double>();
    B.boys2 = boys2;
    B.nao = nao;
    return B;
  }
  // Grow the scratch buffer, ordered on the calling stream: the old buffer is
  // released after the work already queued on `st` (calls on one context are
  // ordered on one stream by contract).
  int ensure_scratch(size_t bytes, cudaStream_t st) {
    if (scratch.bytes >= bytes) return LTJK_OK;
    return scratch.alloc(bytes + bytes / 4, st);
  }
};

namespace {

struct HostPairs {
  std::vector<int2> sh;
  std::vector<int> cls, pp0, npp;
  std::vector<double> zeta, izeta, P, pref, a, b;
  std::vector<float2> pp2;  // double-float copies, 8 per primitive pair
  std::vector<double> ppg;  // specialised kernel: kPrimDf per primitive pair
  std::vector<float2> ppg2;
};

void build_pairs(const ltjk_ctx &c, const std::vector<int2> &order, HostPairs &hp) {
  const double pi = 3.14159265358979323846;
  const double s2pi52 = std::sqrt(2.0 * std::pow(pi, 2.5));
  hp = HostPairs{};
  for (const int2 &pr : order) {
    const int sa = pr.x, sb = pr.y;
    const double *A = &c.coords[3 * c.sh_atom[sa]], *B = &c.coords[3 * c.sh_atom[sb]];
    double AB2 = 0.0;
    for (int x = 0; x < 3; ++x) AB2 += (A[x] - B[x]) * (A[x] - B[x]);
    hp.sh.push_back(pr);
    hp.pp0.push_back((int)hp.zeta.size());
    int kept = 0;
    for (int i = 0; i < c.sh_nprim[sa]; ++i)
      for (int j = 0; j < c.sh_nprim[sb]; ++j) {
        const double al = c.exps[c.sh_p0[sa] + i], be = c.exps[c.sh_p0[sb] + j];
        const double ca = c.ncoef[c.sh_p0[sa] + i], cb = c.ncoef[c.sh_p0[sb] + j];
        const double z = al + be;
        const double kab = std::exp(-al * be / z * AB2);
        if (kab * std::fabs(ca * cb) < kPrimPairDrop) continue;
        hp.zeta.push_back(z);
        hp.izeta.push_back(1.0 / z);
        for (int x = 0; x < 3; ++x) hp.P.push_back((al * A[x] + be * B[x]) / z);
        hp.pref.push_back(s2pi52 * kab * ca * cb / z);
        hp.a.push_back(al);
        hp.b.push_back(be);
        const double Pv[3] = {(al * A[0] + be * B[0]) / z, (al * A[1] + be * B[1]) / z,
                              (al * A[2] + be * B[2]) / z};
        for (double v : {z, 1.0 / z, Pv[0], Pv[1], Pv[2], s2pi52 * kab * ca * cb / z, al, be})
          hp.pp2.push_back(split2(v));
        for (double v : {z, 1.0 / z, Pv[0], Pv[1], Pv[2], Pv[0] - A[0], Pv[1] - A[1], Pv[2] - A[2],
                         s2pi52 * kab * ca * cb / z}) {
          hp.ppg.push_back(v);
          hp.ppg2.push_back(split2(v));
        }
        ++kept;
      }
    hp.npp.push_back(kept);
  }
}

int upload_pairs(ltjk_ctx &c, const HostPairs &hp) {
  int rc;
  std::vector<int> pair_shx;
  if ((rc = c.d_pair_sh.upload(hp.sh)) || (rc = c.d_pair_pp0.upload(hp.pp0)) ||
      (rc = c.d_pair_npp.upload(hp.npp)) || (rc = c.d_pp_zeta.upload(hp.zeta)) ||
      (rc = c.d_pp_izeta.upload(hp.izeta)) || (rc = c.d_pp_P.upload(hp.P)) ||
      (rc = c.d_pp_pref.upload(hp.pref)) || (rc = c.d_pp_a.upload(hp.a)) ||
      (rc = c.d_pp_b.upload(hp.b)) || (rc = c.d_pp2.upload(hp.pp2)) || (rc = c.d_ppg.upload(hp.ppg)) ||
      (rc = c.d_ppg2.upload(hp.ppg2)))
    return rc;
  return LTJK_OK;
}

// Evaluate contracted blocks (pair i | pair j) for a list of (i, j) in `prec`.
int store_blocks(ltjk_ctx &c, const std::vector<std::pair<int, int>> &qs, int prec,
                 std::vector<long long> &offsets, double *d_out, cudaStream_t st) {
  const ProgramSet *ps;
  int rc = program_set(&ps);
  if (rc) return rc;
  // group by class
  std::map<int, std::vector<int>> by_class;
  offsets.assign(qs.size(), 0);
  long long off = 0;
  for (size_t k = 0; k < qs.size(); ++k) {
    const int2 ab = c.pair_sh[qs[k].first], cd = c.pair_sh[qs[k].second];
    const int qi = quartet_index(c.sh_l[ab.x], c.sh_l[ab.y], c.sh_l[cd.x], c.sh_l[cd.y], 0);
    by_class[qi].push_back((int)k);
    offsets[k] = off;
    off += ps->progs[qi].nout;  // the whole value block, its tiles at their own offsets
  }
  DevBasis B = c.basis();
  for (auto &kv : by_class) {
    const ClassProg &p = ps->progs[kv.first];
    std::vector<WorkItem> items;
    std::vector<long long> ioff;
    for (int k : kv.second) {
      items.push_back(WorkItem{qs[k].first, qs[k].second, 1, 0});  // absolute ket pair
      ioff.push_back(offsets[k]);
    }
    DevBuf d_items, d_off;
    if ((rc = d_items.upload(items)) || (rc = d_off.upload(ioff))) return rc;
    JKArgs a{};
    a.out = d_out;
    a.out_off = d_off.as<long long>();
    if (prec == LTJK_FP64_NATIVE || (prec == LTJK_FP64 && ieee64_class(p.la, p.lb, p.lc, p.ld))) {
      ClassLaunch cl = make_launch(p, sizeof(double));
      rc = launch_class<double, kStore>(c.progs, cl,
                                        single_job(B, a, d_items.as<WorkItem>(), (int)items.size()), st);
    } else if (prec == LTJK_FP64) {
      ClassLaunch cl = make_launch(p, sizeof(dflt));
      rc = launch_class<dflt, kStore>(c.progs, cl,
                                      single_job(B, a, d_items.as<WorkItem>(), (int)items.size()), st);
    } else {
      ClassLaunch cl = make_launch(p, sizeof(float));
      rc = launch_class<float, kStore>(c.progs, cl,
                                       single_job(B, a, d_items.as<WorkItem>(), (int)items.size()), st);
    }
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(st));  // the temporary item lists die here
  }
  return LTJK_OK;
}

// Flop model of a class (per contracted quartet with npq primitive quartets).
// (npq primitive quartets over nq contracted quartets): per primitive quartet
// the vertical recurrence, the Boys function and set-up, the accumulation;
// per contracted quartet the horizontal recurrence.
double class_flops(const ClassProg &p, long long npq, long long nq) {
  const double boys = 40.0;
  return npq * (p.vrr_flops + boys + 30.0 + 2.0 * p.nacc) + nq * p.hrr_flops;
}

int build_work(ltjk_ctx &c) {
  const ProgramSet *ps;
  int rc = program_set(&ps);
  if (rc) return rc;
  const double tau = c.opts.schwarz_tau;
  const bool mixed = c.opts.precision == LTJK_MIXED;
  const double tmix = c.opts.mixed_tau;
  c.work.clear();
  c.stats.quartets_total = 0;
  c.stats.quartets_kept = 0;
  c.stats.quartets_fp64 = 0;
  c.stats.prim_quartets_kept = 0;
  c.stats.cart_integrals_kept = 0;
  c.stats.eri_flops_per_build = 0;
  c.stats.eri_flops_fp64 = 0;
  c.stats.cart_integrals_fp64 = 0;
  c.stats.grad_eri_flops = 0;
  c.stats.grad_eri_flops_fp64 = 0;
  std::vector<int> npp_host(c.npairs);
  {
    // primitive pair counts are needed for the statistics
    std::vector<int> tmp(c.npairs);
    CUDA_TRY(cudaMemcpy(tmp.data(), c.d_pair_npp.p, sizeof(int) * c.npairs, cudaMemcpyDeviceToHost));
    npp_host = tmp;
  }
  for (int X = 0; X < kNumPairClass; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      const int xb = c.class_begin[X], xe = c.class_begin[X + 1];
      const int yb = c.class_begin[Y], ye = c.class_begin[Y + 1];
      if (xb == xe || yb == ye) continue;
      auto cw = std::make_unique<ClassWork>();
      cw->X = X;
      cw->Y = Y;
      const int2 s0 = c.pair_sh[xb], t0 = c.pair_sh[yb];
      cw->la = c.sh_l[s0.x];
      cw->lb = c.sh_l[s0.y];
      cw->lc = c.sh_l[t0.x];
      cw->ld = c.sh_l[t0.y];
      cw->ket_base = yb;
      const ClassProg &p = ps->progs[quartet_index(cw->la, cw->lb, cw->lc, cw->ld, 0)];
      const ClassProg &pd = ps->progs[quartet_index(cw->la, cw->lb, cw->lc, cw->ld, 1)];
      // Schwarz-kept ket prefix of every bra pair, split FP64-class / FP32
      std::vector<int> keep(xe - xb), n64v(xe - xb);
      long long tot64 = 0, tot32 = 0;
      for (int i = xb; i < xe; ++i) {
        const double qi = c.pair_Q[i];
        int nj = ye - yb;
        if (X == Y) nj = i - xb + 1;
        c.stats.quartets_total += nj;
        // prefix of kets with Q_i Q_j >= tau (Q sorted descending)
        int lo = 0, hi = nj;
        while (lo < hi) {
          int mid = (lo + hi) / 2;
          if (qi * c.pair_Q[yb + mid] >= tau) lo = mid + 1; else hi = mid;
        }
        const int nkeep = lo;
        int n64 = nkeep;
        if (mixed) {
          lo = 0;
          hi = nkeep;
          while (lo < hi) {
            int mid = (lo + hi) / 2;
            if (qi * c.pair_Q[yb + mid] > tmix) lo = mid + 1; else hi = mid;
          }
          n64 = lo;
        }
        keep[i - xb] = nkeep;
        n64v[i - xb] = n64;
        tot64 += n64;
        tot32 += nkeep - n64;
        c.stats.quartets_kept += nkeep;
        c.stats.quartets_fp64 += n64;
        long long npq = 0, npq64 = 0;
        for (int j = 0; j < nkeep; ++j) {
          npq += (long long)npp_host[i] * npp_host[yb + j];
          if (j == n64 - 1) npq64 = npq;
        }
        c.stats.prim_quartets_kept += npq;
        const long long nint = (long long)ncart(cw->la) * ncart(cw->lb) * ncart(cw->lc) * ncart(cw->ld);
        c.stats.cart_integrals_kept += (long long)nkeep * nint;
        c.stats.cart_integrals_fp64 += (long long)n64 * nint;
        c.stats.eri_flops_per_build += class_flops(p, npq, nkeep);
        c.stats.eri_flops_fp64 += class_flops(p, npq64, n64);
        c.stats.grad_eri_flops += class_flops(pd, npq, nkeep);
        c.stats.grad_eri_flops_fp64 += class_flops(pd, npq64, n64);
      }
      // kets per work item: small enough that a class yields at least
      // kTargetItems items (heavy classes have few quartets), at most kKetChunk
      // (the class-specialised kernel runs one ket per lane: up to 32 per item)
      const int cap = gen_class(cw->la, cw->lb, cw->lc, cw->ld) ? kGenKetChunk : kKetChunk;
      auto chunk_of = [cap](long long total) {
        return (int)std::max<long long>(1, std::min<long long>(cap, (total + kTargetItems - 1) / kTargetItems));
      };
      const int ch64 = chunk_of(tot64), ch32 = chunk_of(tot32);
      std::vector<WorkItem> i64, i32;
      for (int i = xb; i < xe; ++i) {
        const int nkeep = keep[i - xb], n64 = n64v[i - xb];
        for (int k = 0; k < n64; k += ch64) i64.push_back({i, yb + k, std::min(ch64, n64 - k), 0});
        for (int k = n64; k < nkeep; k += ch32) i32.push_back({i, yb + k, std::min(ch32, nkeep - k), 0});
      }
      if ((rc = cw->items64.upload(i64)) || (rc = cw->items32.upload(i32))) return rc;
      cw->n64 = (int)i64.size();
      cw->n32 = (int)i32.size();
      c.work.push_back(std::move(cw));
    }
  return LTJK_OK;
}


// Device scratch of one J/K build of nd densities: two density copies, the J
// and K accumulators (q-innermost), plus FP32 copies in mixed precision, plus
// one power-of-two scale per density.
size_t jk_scratch_bytes(const ltjk_ctx *c, int nd) {
  const size_t n = (size_t)c->nao * c->nao * nd;
  return 4 * n * sizeof(double) + (c->opts.precision == LTJK_MIXED ? 2 * n * sizeof(float) : 0) +
         (c->ieee_copies ? 2 * n * sizeof(double) : 0) + (size_t)nd * sizeof(double);
}

// Enqueue the per-density scales, the layout transposes and the accumulator
// clear of one J/K build whose scratch starts at `base` (jk_scratch_bytes
// bytes); the kernel arguments go to *out.  Each density is scaled by the
// power of two that brings its largest element into [1/2, 1): the build is
// linear in D and the scaling is exact, so the double-float and binary32
// copies keep their full relative precision whatever the magnitude of D
// (binary32 words alone would flush elements below 2^-126 to zero).
int jk_prologue(const ltjk_ctx *c, const double *D, void *base, int nd, bool wantJ, bool wantK,
                cudaStream_t st, JKArgs *out) {
  const size_t n = (size_t)c->nao * c->nao * nd;
  double *A = static_cast<double *>(base), *Bq = A + n, *Jq = Bq + n, *Kq = Jq + n;
  const bool native = c->opts.precision == LTJK_FP64_NATIVE;
  const bool mixed = c->opts.precision == LTJK_MIXED;
  float *D32 = mixed ? reinterpret_cast<float *>(Kq + n) : nullptr;
  float *S32 = mixed ? D32 + n : nullptr;
  double *D64 = c->ieee_copies ? Kq + n + (mixed ? n : 0) : nullptr;  // beside the double-float copies
  double *S64 = c->ieee_copies ? D64 + n : nullptr;
  double *scale = Kq + n + (mixed ? n : 0) + (c->ieee_copies ? 2 * n : 0);
  JKArgs a{};
  if (native) {
    a.D = A;
    a.S = Bq;
  } else {
    a.D2 = reinterpret_cast<dflt *>(A);
    a.S2 = reinterpret_cast<dflt *>(Bq);
    a.D = D64;
    a.S = S64;
  }
  a.D32 = D32;
  a.S32 = S32;
  a.J = wantJ ? Jq : nullptr;
  a.K = wantK ? Kq : nullptr;
  a.nd = nd;
  a.scale = scale;
  density_scales<<<nd, 256, 0, st>>>(D, (size_t)c->nao * c->nao, scale);
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16);
  to_qinner<<<blocks, 256, 0, st>>>(D, native ? A : D64, native ? Bq : S64, D32, S32, nd,
                                    c->nao, native ? nullptr : reinterpret_cast<dflt *>(A),
                                    native ? nullptr : reinterpret_cast<dflt *>(Bq), scale);
  CUDA_TRY(cudaGetLastError());
  g_launches += 2;
  CUDA_TRY(cudaMemsetAsync(Jq, 0, 2 * n * sizeof(double), st));
  *out = a;
  return LTJK_OK;
}

// Enqueue the epilogue of one J/K build: J = Jh + Jh^T and K, unscaled, in
// the caller's [nd][N][N] layout.
int jk_epilogue(const ltjk_ctx *c, const JKArgs &a, double *J, double *K, cudaStream_t st) {
  const size_t n = (size_t)c->nao * c->nao * a.nd;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16);
  from_qinner<<<blocks, 256, 0, st>>>(a.J, a.K, J, K, a.nd, c->nao, a.scale);
  CUDA_TRY(cudaGetLastError());
  g_launches += 1;
  return LTJK_OK;
}

// The class launches of one pass (J/K or gradient) over a context's work
// lists: FP64-class items in double-float (native FP64 on request), FP32 items
// (mixed precision) in float.
template <int MODE>
int launch_classes(ltjk_ctx *ctx, const JKArgs &a, cudaStream_t st) {
  const ProgramSet *ps;
  int rc = program_set(&ps);
  if (rc) return rc;
  const bool native = ctx->opts.precision == LTJK_FP64_NATIVE;
  const DevBasis B = ctx->basis();
  // fork: the class launches are independent (they only add into J, K or the
  // gradient), so they run on the context's side streams concurrently, which
  // keeps the GPU full while a heavy class with few work items runs
  CUDA_TRY(cudaEventRecord(ctx->fork_ev, st));
  for (int k = 0; k < kSideStreams; ++k) CUDA_TRY(cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0));
  int next = 0;
  for (auto &w : ctx->work) {
    const ClassProg &p = ps->progs[quartet_index(w->la, w->lb, w->lc, w->ld, MODE == kGrad)];
    if (w->n64) {
      cudaStream_t s2 = ctx->side[next++ % kSideStreams];
      const JobTable T = single_job(B, a, w->items64.as<WorkItem>(), w->n64);
      const bool ieee = native || ieee64_class(p.la, p.lb, p.lc, p.ld);
      if (MODE == kJK)
        rc = ieee ? launch_jk<double>(p, ctx->progs, T, s2) : launch_jk<dflt>(p, ctx->progs, T, s2);
      else
        rc = ieee ? launch_class<double, MODE>(ctx->progs, grad_launch(p, sizeof(double)), T, s2)
                  : launch_class<dflt, MODE>(ctx->progs, grad_launch(p, sizeof(dflt)), T, s2);
      if (rc) return rc;
    }
    if (w->n32) {
      cudaStream_t s2 = ctx->side[next++ % kSideStreams];
      const JobTable T = single_job(B, a, w->items32.as<WorkItem>(), w->n32);
      rc = MODE == kJK ? launch_jk<float>(p, ctx->progs, T, s2)
                       : launch_class<float, MODE>(ctx->progs, grad_launch(p, sizeof(float)), T, s2);
      if (rc) return rc;
    }
  }
  // join
  for (int k = 0; k < kSideStreams; ++k) {
    CUDA_TRY(cudaEventRecord(ctx->join_ev[k], ctx->side[k]));
    CUDA_TRY(cudaStreamWaitEvent(st, ctx->join_ev[k], 0));
  }
  return LTJK_OK;
}

}  // namespace

extern "C" {

const char *ltjk_last_error(void) { return last_error(); }

int ltjk_launch_count(unsigned long long *count) {
  if (!count) return set_error(LTJK_EINVAL, "launch_count: null argument");
  *count = g_launches.load();
  return LTJK_OK;
}
int ltjk_version(void) { return 100; }

static_assert(kMaxPrim == LTJK_MAX_PRIM, "primitive limit of the header and the kernels");

int ltjk_context_create(const ltjk_basis *bs, const ltjk_opts *opts, ltjk_ctx **out) {
  if (!bs || !opts || !out) return set_error(LTJK_EINVAL, "context_create: null argument");
  *out = nullptr;
  if (bs->natoms <= 0 || bs->nshells <= 0 || !bs->coords_host || !bs->shell_atom_host ||
      !bs->shell_l_host || !bs->shell_nprim_host || !bs->exps_host || !bs->coefs_host)
    return set_error(LTJK_EINVAL, "context_create: empty or incomplete basis");
  if (opts->precision != LTJK_FP64 && opts->precision != LTJK_MIXED &&
      opts->precision != LTJK_FP64_NATIVE)
    return set_error(LTJK_EINVAL,
                     "context_create: precision must be LTJK_FP64, LTJK_MIXED or LTJK_FP64_NATIVE");
  if (!(opts->schwarz_tau >= 0) || !(opts->mixed_tau >= 0))
    return set_error(LTJK_EINVAL, "context_create: thresholds must be >= 0");
  auto c = std::make_unique<ltjk_ctx>();
  c->opts = *opts;
  c->device = opts->device;
  c->natoms = bs->natoms;
  c->nshells = bs->nshells;
  c->coords.assign(bs->coords_host, bs->coords_host + 3 * bs->natoms);
  int np = 0;
  for (int s = 0; s < bs->nshells; ++s) {
    const int l = bs->shell_l_host[s], n = bs->shell_nprim_host[s], at = bs->shell_atom_host[s];
    if (l < 0) return set_error(LTJK_EINVAL, "shell %d: negative angular momentum", s);
    if (l > kMaxL)
      return set_error(LTJK_EUNSUPPORTED, "shell %d: l = %d above LTJK_MAX_L = %d", s, l, kMaxL);
    if (n < 1 || n > kMaxPrim) return set_error(LTJK_EINVAL, "shell %d: nprim %d not in 1..%d", s, n, kMaxPrim);
    if (at < 0 || at >= bs->natoms) return set_error(LTJK_EINVAL, "shell %d: atom %d out of range", s, at);
    c->sh_l.push_back(l);
    c->sh_atom.push_back(at);
    c->sh_nprim.push_back(n);
    c->sh_p0.push_back(np);
    c->sh_ao.push_back(c->nao);
    c->nao += ncart(l);
    np += n;
    if (ieee64_class(l, 0, 0, 0) && c->opts.precision != LTJK_FP64_NATIVE) c->ieee_copies = true;
  }
  c->exps.assign(bs->exps_host, bs->exps_host + np);
  for (double e : c->exps)
    if (!(e > 0) || !std::isfinite(e)) return set_error(LTJK_EINVAL, "non-positive primitive exponent");
  for (int t = 0; t < 3 * bs->natoms; ++t)
    if (!std::isfinite(c->coords[t])) return set_error(LTJK_EINVAL, "non-finite coordinate");
  c->ncoef.resize(np);
  for (int s = 0; s < c->nshells; ++s)
    normalise_shell(c->sh_l[s], c->sh_nprim[s], &c->exps[c->sh_p0[s]], bs->coefs_host + c->sh_p0[s],
                    &c->ncoef[c->sh_p0[s]]);
  // the basis is checked on the host before the first CUDA call
  CUDA_TRY(cudaSetDevice(c->device));
  int rc;
  if ((rc = device_programs(c->device, &c->progs, &c->boys, &c->boys2))) return rc;
  CUDA_TRY(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
  for (int k = 0; k < kSideStreams; ++k) {
    CUDA_TRY(cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming));
  }
  std::vector<double> ctr(3 * c->nshells);
  for (int s = 0; s < c->nshells; ++s)
    for (int x = 0; x < 3; ++x) ctr[3 * s + x] = c->coords[3 * c->sh_atom[s] + x];
  std::vector<float2> ctr2;
  for (double v : ctr) ctr2.push_back(split2(v));
  if ((rc = c->d_ctr.upload(ctr)) || (rc = c->d_ctr2.upload(ctr2)) || (rc = c->d_l.upload(c->sh_l)) ||
      (rc = c->d_ao.upload(c->sh_ao)) ||
      (rc = c->d_atom.upload(c->sh_atom)))
    return rc;
  // canonical pairs grouped by class: l_a >= l_b, and a >= b when l_a == l_b
  std::vector<std::vector<int2>> by_class(kNumPairClass);
  for (int a = 0; a < c->nshells; ++a)
    for (int b = 0; b < c->nshells; ++b) {
      const int la = c->sh_l[a], lb = c->sh_l[b];
      if (la < lb || (la == lb && a < b)) continue;
      by_class[pair_class(la, lb)].push_back(make_int2(a, b));
    }
  std::vector<int2> order;
  for (auto &v : by_class) order.insert(order.end(), v.begin(), v.end());
  c->npairs = (int)order.size();
  HostPairs hp;
  build_pairs(*c, order, hp);
  c->pair_sh = order;
  if ((rc = upload_pairs(*c, hp))) return rc;
  // Schwarz factors from the diagonal quartets (ab|ab), evaluated in FP64
  {
    std::vector<std::pair<int, int>> qs;
    for (int i = 0; i < c->npairs; ++i) qs.push_back({i, i});
    const ProgramSet *ps;
    if ((rc = program_set(&ps))) return rc;
    long long total = 0;
    for (int i = 0; i < c->npairs; ++i) {
      const int2 ab = order[i];
      total += (long long)ncart(c->sh_l[ab.x]) * ncart(c->sh_l[ab.y]) * ncart(c->sh_l[ab.x]) *
               ncart(c->sh_l[ab.y]);
    }
    DevBuf d_out;
    if ((rc = d_out.alloc(sizeof(double) * std::max<long long>(total, 1)))) return rc;
    std::vector<long long> offs;
    // on a private highest-priority stream: a context created while other
    // work runs (a serving frontend) does not wait behind that work's blocks
    int plo = 0, phi = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&plo, &phi));
    cudaStream_t cst = nullptr;
    CUDA_TRY(cudaStreamCreateWithPriority(&cst, cudaStreamNonBlocking, phi));
    rc = store_blocks(*c, qs, LTJK_FP64_NATIVE, offs, d_out.as<double>(), cst);
    cudaStreamSynchronize(cst);
    cudaStreamDestroy(cst);
    if (rc) return rc;
    std::vector<double> blocks(total);
    CUDA_TRY(cudaMemcpy(blocks.data(), d_out.p, sizeof(double) * total, cudaMemcpyDeviceToHost));
    c->pair_Q.assign(c->npairs, 0.0);
    for (int i = 0; i < c->npairs; ++i) {
      const int na = ncart(c->sh_l[order[i].x]), nb = ncart(c->sh_l[order[i].y]);
      double m = 0.0;
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) {
          const double v = std::fabs(blocks[offs[i] + ((x * nb + y) * na + x) * nb + y]);
          m = std::max(m, v);
        }
      c->pair_Q[i] = std::sqrt(m);
    }
  }
  // sort each class by Q descending and rebuild the pair data in that order
  {
    std::vector<int2> sorted;
    std::vector<double> qsorted;
    c->class_begin.assign(kNumPairClass + 1, 0);
    int base = 0;
    for (int X = 0; X < kNumPairClass; ++X) {
      const int n = (int)by_class[X].size();
      std::vector<int> idx(n);
      for (int k = 0; k < n; ++k) idx[k] = base + k;
      std::stable_sort(idx.begin(), idx.end(), [&](int u, int v) { return c->pair_Q[u] > c->pair_Q[v]; });
      c->class_begin[X] = (int)sorted.size();
      for (int k : idx) {
        sorted.push_back(order[k]);
        qsorted.push_back(c->pair_Q[k]);
      }
      base += n;
    }
    c->class_begin[kNumPairClass] = (int)sorted.size();
    c->pair_sh = sorted;
    c->pair_Q = qsorted;
    build_pairs(*c, sorted, hp);
    if ((rc = upload_pairs(*c, hp))) return rc;
    for (int i = 0; i < c->npairs; ++i) c->pair_of[{sorted[i].x, sorted[i].y}] = i;
  }
  if ((rc = build_work(*c))) return rc;
  c->stats.nao = c->nao;
  c->stats.nshells = c->nshells;
  c->stats.npairs = c->npairs;
  *out = c.release();
  return LTJK_OK;
}

int ltjk_context_destroy(ltjk_ctx *ctx) {
  if (!ctx) return set_error(LTJK_EINVAL, "context_destroy: null context");
  cudaSetDevice(ctx->device);
  // the context's own streams; work the caller queued on its streams must be
  // complete (or ordered before the legacy stream) by contract
  for (int k = 0; k < kSideStreams; ++k)
    if (ctx->side[k]) cudaStreamSynchronize(ctx->side[k]);
  delete ctx;
  return LTJK_OK;
}

int ltjk_nao(const ltjk_ctx *ctx, int *nao) {
  if (!ctx || !nao) return set_error(LTJK_EINVAL, "nao: null argument");
  *nao = ctx->nao;
  return LTJK_OK;
}

int ltjk_nsph(const ltjk_ctx *ctx, int *nsph) {
  if (!ctx || !nsph) return set_error(LTJK_EINVAL, "nsph: null argument");
  int n = 0;
  for (int l : ctx->sh_l) n += 2 * l + 1;
  *nsph = n;
  return LTJK_OK;
}

int ltjk_sph_transform(ltjk_ctx *ctx, int direction, int ndens, const double *A, double *B,
                       ltjk_stream stream) {
  if (!ctx || !A || !B) return set_error(LTJK_EINVAL, "sph_transform: null argument");
  if ((direction != 0 && direction != 1) || ndens < 1 || ndens > 4096)
    return set_error(LTJK_EINVAL, "sph_transform: direction must be 0 or 1 and 1 <= ndens <= 4096");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int Nc = ctx->nao;
  int rc;
  if (ctx->nsph == 0) {
    // T, block diagonal: real solid harmonics of each shell in terms of its
    // Cartesian components (every component normalised as x^l); p keeps the
    // Cartesian order x, y, z; d and f in the order m = -l..l.
    int Ns = 0;
    for (int l : ctx->sh_l) Ns += 2 * l + 1;
    std::vector<double> T((size_t)Ns * Nc, 0.0);
    const double r3 = std::sqrt(3.0);
    int row = 0;
    for (int sh = 0; sh < ctx->nshells; ++sh) {
      const int l = ctx->sh_l[sh], c0 = ctx->sh_ao[sh];
      auto at = [&](int r, int c) -> double & { return T[(size_t)(row + r) * Nc + c0 + c]; };
      if (l == 0) {
        at(0, 0) = 1.0;
      } else if (l == 1) {
        for (int k = 0; k < 3; ++k) at(k, k) = 1.0;
      } else if (l == 2) {  // components xx, xy, xz, yy, yz, zz
        at(0, 1) = r3;                   // xy
        at(1, 4) = r3;                   // yz
        at(2, 0) = -0.5;                 // (2 zz - xx - yy) / 2
        at(2, 3) = -0.5;
        at(2, 5) = 1.0;
        at(3, 2) = r3;                   // xz
        at(4, 0) = 0.5 * r3;             // (xx - yy) sqrt3 / 2
        at(4, 3) = -0.5 * r3;
      } else if (l == 3) {
        // components xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz; m = -3..3:
        //   sqrt(5/8) (3 xxy - yyy), sqrt15 xyz, sqrt(3/8) (4 yzz - xxy - yyy),
        //   (2 zzz - 3 xxz - 3 yyz) / 2, sqrt(3/8) (4 xzz - xxx - xyy),
        //   sqrt15 / 2 (xxz - yyz), sqrt(5/8) (xxx - 3 xyy)
        // (each the unit-norm multiple of its harmonic polynomial, with the
        // one-centre overlap of x^a y^b z^c normalised as x^3)
        const double c58 = std::sqrt(5.0 / 8.0), c38 = std::sqrt(3.0 / 8.0), r15 = std::sqrt(15.0);
        at(0, 1) = 3.0 * c58;
        at(0, 6) = -c58;
        at(1, 4) = r15;
        at(2, 8) = 4.0 * c38;
        at(2, 1) = -c38;
        at(2, 6) = -c38;
        at(3, 9) = 1.0;
        at(3, 2) = -1.5;
        at(3, 7) = -1.5;
        at(4, 5) = 4.0 * c38;
        at(4, 0) = -c38;
        at(4, 3) = -c38;
        at(5, 2) = 0.5 * r15;
        at(5, 7) = -0.5 * r15;
        at(6, 0) = c58;
        at(6, 3) = -3.0 * c58;
      } else {
        return set_error(LTJK_EUNSUPPORTED, "sph_transform: l = %d", l);
      }
      row += 2 * l + 1;
    }
    if ((rc = ctx->d_sph.upload(T))) return rc;
    ctx->nsph = Ns;
  }
  const int Ns = ctx->nsph;
  const double *T = ctx->d_sph.as<double>();
  if ((rc = ctx->ensure_scratch((size_t)ndens * Ns * Nc * sizeof(double), st))) return rc;
  double *X = ctx->scratch.as<double>();
  const dim3 thr(16, 16);
  if (direction == 0) {
    // X[q] = T A[q] ([Ns][Nc] x [Nc][Nc]); B[q] = X[q] T^T ([Ns][Nc] x [Nc][Ns])
    gemm_f64<false><<<dim3((Nc + 15) / 16, (Ns + 15) / 16, ndens), thr, 0, st>>>(
        T, 0, A, (long long)Nc * Nc, X, (long long)Ns * Nc, Ns, Nc, Nc, Nc, Nc, Nc);
    gemm_f64<true><<<dim3((Ns + 15) / 16, (Ns + 15) / 16, ndens), thr, 0, st>>>(
        X, (long long)Ns * Nc, T, 0, B, (long long)Ns * Ns, Ns, Ns, Nc, Nc, Nc, Ns);
  } else {
    // X[q] = T^T A[q] ([Nc][Ns] x [Ns][Ns]); B[q] = X[q] T ([Nc][Ns] x [Ns][Nc])
    gemm_f64<false, true><<<dim3((Ns + 15) / 16, (Nc + 15) / 16, ndens), thr, 0, st>>>(
        T, 0, A, (long long)Ns * Ns, X, (long long)Nc * Ns, Nc, Ns, Ns, Nc, Ns, Ns);
    gemm_f64<false><<<dim3((Nc + 15) / 16, (Nc + 15) / 16, ndens), thr, 0, st>>>(
        X, (long long)Nc * Ns, T, 0, B, (long long)Nc * Nc, Nc, Nc, Ns, Ns, Nc, Nc);
  }
  CUDA_TRY(cudaGetLastError());
  g_launches += 2;
  return LTJK_OK;
}

int ltjk_context_stats(const ltjk_ctx *ctx, ltjk_ctx_stats *out) {
  if (!ctx || !out) return set_error(LTJK_EINVAL, "context_stats: null argument");
  *out = ctx->stats;
  size_t b = 0;
  for (const DevBuf *d : {&ctx->d_ctr, &ctx->d_l, &ctx->d_ao, &ctx->d_atom, &ctx->d_pair_sh,
                          &ctx->d_pair_pp0, &ctx->d_pair_npp, &ctx->d_pp_zeta, &ctx->d_pp_izeta,
                          &ctx->d_pp_P, &ctx->d_pp_pref, &ctx->d_pp_a, &ctx->d_pp_b, &ctx->scratch})
    b += d->bytes;
  for (auto &w : ctx->work) b += w->items64.bytes + w->items32.bytes;
  out->device_bytes = b;
  return LTJK_OK;
}

int ltjk_schwarz(const ltjk_ctx *ctx, double *Q_host) {
  if (!ctx || !Q_host) return set_error(LTJK_EINVAL, "schwarz: null argument");
  const int ns = ctx->nshells;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      auto it = ctx->pair_of.find({a, b});
      if (it == ctx->pair_of.end()) it = ctx->pair_of.find({b, a});
      Q_host[a * ns + b] = ctx->pair_Q[it->second];
    }
  return LTJK_OK;
}

int ltjk_laplace_quadrature(double xmin, double xmax, int n, double *t_host, double *w_host,
                            double *max_rel_err) {
  return laplace_quadrature(xmin, xmax, n, t_host, w_host, max_rel_err);
}

int ltjk_laplace_minimax(double xmin, double xmax, int n, double *t_host, double *w_host,
                         double *max_rel_err, int *converged) {
  return laplace_minimax(xmin, xmax, n, t_host, w_host, max_rel_err, converged);
}

int ltjk_laplace_shift(int n, const double *t_host, const double *w_host, double omega,
                       double *w_shifted_host) {
  if (n < 1 || !t_host || !w_host || !w_shifted_host || !std::isfinite(omega))
    return set_error(LTJK_EINVAL, "laplace_shift: bad argument");
  for (int q = 0; q < n; ++q) w_shifted_host[q] = w_host[q] * std::exp(omega * t_host[q]);
  return LTJK_OK;
}

int ltjk_jk_build(ltjk_ctx *ctx, int ndens, const double *D, double *J, double *K,
                  ltjk_stream stream) {
  if (!ctx || !D) return set_error(LTJK_EINVAL, "jk_build: null context or density");
  if (ndens < 1 || ndens > 4096) return set_error(LTJK_EINVAL, "jk_build: ndens %d not in 1..4096", ndens);
  if (!J && !K) return LTJK_OK;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = ctx->ensure_scratch(jk_scratch_bytes(ctx, ndens), st);
  if (rc) return rc;
  JKArgs a;
  if ((rc = jk_prologue(ctx, D, ctx->scratch.p, ndens, J != nullptr, K != nullptr, st, &a))) return rc;
  if ((rc = launch_classes<kJK>(ctx, a, st))) return rc;
  return jk_epilogue(ctx, a, J, K, st);
}

// F = cJ J[D] + cK K[D] into F ([ndens][N][N], device), scratch at `base`
// (jk_scratch_bytes bytes).
static int jk_fock_into(ltjk_ctx *ctx, int ndens, const double *D, double cJ, double cK, double *F,
                        void *base, cudaStream_t st) {
  const size_t n = (size_t)ctx->nao * ctx->nao * ndens;
  if (cJ == 0.0 && cK == 0.0) {
    CUDA_TRY(cudaMemsetAsync(F, 0, n * sizeof(double), st));
    return LTJK_OK;
  }
  JKArgs a;
  int rc;
  if ((rc = jk_prologue(ctx, D, base, ndens, cJ != 0.0, cK != 0.0, st, &a))) return rc;
  if ((rc = launch_classes<kJK>(ctx, a, st))) return rc;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16);
  from_qinner_fock<<<blocks, 256, 0, st>>>(a.J, a.K, F, ndens, ctx->nao, a.scale, cJ, cK);
  CUDA_TRY(cudaGetLastError());
  g_launches += 1;
  return LTJK_OK;
}

int ltjk_jk_fock(ltjk_ctx *ctx, int ndens, const double *D, double cJ, double cK, double *F,
                 ltjk_stream stream) {
  if (!ctx || !D || !F) return set_error(LTJK_EINVAL, "jk_fock: null argument");
  if (ndens < 1 || ndens > 4096) return set_error(LTJK_EINVAL, "jk_fock: ndens %d not in 1..4096", ndens);
  if (!std::isfinite(cJ) || !std::isfinite(cK)) return set_error(LTJK_EINVAL, "jk_fock: non-finite coefficient");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = ctx->ensure_scratch(jk_scratch_bytes(ctx, ndens), st);
  if (rc) return rc;
  return jk_fock_into(ctx, ndens, D, cJ, cK, F, ctx->scratch.p, st);
}

int ltjk_jk_energy(ltjk_ctx *ctx, int nterms, const double *P, const double *Q, double cJ,
                   double cK, double *F, double *E, ltjk_stream stream) {
  if (!ctx || !P || !Q || !E) return set_error(LTJK_EINVAL, "jk_energy: null argument");
  if (nterms < 1 || nterms > 4096) return set_error(LTJK_EINVAL, "jk_energy: nterms %d not in 1..4096", nterms);
  if (!std::isfinite(cJ) || !std::isfinite(cK)) return set_error(LTJK_EINVAL, "jk_energy: non-finite coefficient");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = (size_t)ctx->nao * ctx->nao * nterms;
  const int nb = (int)std::min<size_t>((n + 4095) / 4096, 1024);
  const size_t jk = (jk_scratch_bytes(ctx, nterms) + 255) / 256 * 256;
  int rc = ctx->ensure_scratch(jk + (F ? 0 : n * sizeof(double)) + nb * sizeof(double), st);
  if (rc) return rc;
  char *base = static_cast<char *>(ctx->scratch.p);
  double *Fb = F ? F : reinterpret_cast<double *>(base + jk);
  double *partial = reinterpret_cast<double *>(base + jk + (F ? 0 : n * sizeof(double)));
  if ((rc = jk_fock_into(ctx, nterms, Q, cJ, cK, Fb, base, st))) return rc;
  dot_partial<<<nb, 256, 0, st>>>(P, Fb, n, partial);
  dot_final<<<1, 32, 0, st>>>(partial, nb, E);
  CUDA_TRY(cudaGetLastError());
  g_launches += 2;
  return LTJK_OK;
}

int ltjk_jk_grad(ltjk_ctx *ctx, int nterms, const double *P, const double *Q, double cJ, double cK,
                 double *grad, ltjk_stream stream) {
  if (!ctx || !P || !Q || !grad) return set_error(LTJK_EINVAL, "jk_grad: null argument");
  if (nterms < 1 || nterms > 4096) return set_error(LTJK_EINVAL, "jk_grad: nterms %d not in 1..4096", nterms);
  for (int s = 0; s < ctx->nshells; ++s)
    if (ctx->sh_l[s] > kMaxLGrad)
      return set_error(LTJK_EUNSUPPORTED, "jk_grad: shell %d has l = %d above LTJK_MAX_L_GRAD = %d", s,
                       ctx->sh_l[s], kMaxLGrad);
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t NN = (size_t)ctx->nao * ctx->nao, n = NN * nterms;
  int rc = ctx->ensure_scratch(4 * n * sizeof(double), st);
  if (rc) return rc;
  double *Pq = ctx->scratch.as<double>(), *Qq = Pq + n;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16);
  to_qinner<<<blocks, 256, 0, st>>>(P, Pq, Qq + n, nullptr, nullptr, nterms, ctx->nao);
  to_qinner<<<blocks, 256, 0, st>>>(Q, Qq, Qq + 2 * n, nullptr, nullptr, nterms, ctx->nao);
  CUDA_TRY(cudaGetLastError());
  g_launches += 2;
  CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(double) * 3 * ctx->natoms, st));
  JKArgs a{};
  a.P = Pq;
  a.Q = Qq;
  a.S = Qq + n;      // P + P^T: the J images of Gamma read 4 words a term instead of 8
  a.D = Qq + 2 * n;  // Q + Q^T
  a.nd = nterms;
  a.cJ = cJ;
  a.cK = cK;
  a.grad = grad;
  return launch_classes<kGrad>(ctx, a, st);
}

int ltjk_pseudo_densities(ltjk_ctx *ctx, int nocc, int nvir, const double *C_occ,
                          const double *C_vir, const double *eps_occ, const double *eps_vir,
                          int npair, const double *X, int nlap, const double *t_host, double *D,
                          ltjk_stream stream) {
  if (!ctx || !C_occ || !C_vir || !eps_occ || !eps_vir || !X || !t_host || !D)
    return set_error(LTJK_EINVAL, "pseudo_densities: null argument");
  if (nocc < 1 || nvir < 1 || npair < 1 || nlap < 1 || (long long)npair * nlap > 4096)
    return set_error(LTJK_EINVAL, "pseudo_densities: bad sizes");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int N = ctx->nao, nq = nlap * npair;
  const size_t ny = (size_t)nq * nocc * nvir, nz = (size_t)nq * nocc * N;
  int rc;
  if (ctx->d_t.bytes < sizeof(double) * nlap &&
      (rc = ctx->d_t.alloc(sizeof(double) * 64 * ((nlap + 63) / 64), st)))
    return rc;
  if ((rc = ctx->ensure_scratch((ny + nz) * sizeof(double), st))) return rc;
  double *Y = ctx->scratch.as<double>(), *Z = Y + ny;
  CUDA_TRY(cudaMemcpyAsync(ctx->d_t.p, t_host, sizeof(double) * nlap, cudaMemcpyHostToDevice, st));
  scale_amplitudes<<<(int)std::min<size_t>((ny + 255) / 256, (size_t)num_sms() * 16), 256, 0, st>>>(
      X, eps_occ, eps_vir, ctx->d_t.as<double>(), Y, nlap, npair, nocc, nvir);
  dim3 thr(16, 16);
  dim3 g1((N + 15) / 16, (nocc + 15) / 16, nq);
  gemm_f64<true><<<g1, thr, 0, st>>>(Y, (long long)nocc * nvir, C_vir, 0, Z, (long long)nocc * N,
                                     nocc, N, nvir, nvir, nvir, N);
  dim3 g2((N + 15) / 16, (N + 15) / 16, nq);
  gemm_f64<false><<<g2, thr, 0, st>>>(C_occ, 0, Z, (long long)nocc * N, D, (long long)N * N, N, N,
                                      nocc, nocc, N, N);
  CUDA_TRY(cudaGetLastError());
  g_launches += 3;
  return LTJK_OK;
}

int ltjk_laplace_fock(ltjk_ctx *ctx, int ndens, const double *J, const double *K, double cJ,
                      double cK, int nl, const double *C_left, int nr, const double *C_right,
                      double *F, ltjk_stream stream) {
  if (!ctx || !J || !K || !C_left || !C_right || !F)
    return set_error(LTJK_EINVAL, "laplace_fock: null argument");
  if (ndens < 1 || ndens > 4096 || nl < 1 || nr < 1)
    return set_error(LTJK_EINVAL, "laplace_fock: bad sizes");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int N = ctx->nao;
  const size_t nm = (size_t)ndens * N * N, nt = (size_t)ndens * N * nr;
  int rc = ctx->ensure_scratch((nm + nt) * sizeof(double), st);
  if (rc) return rc;
  double *M = ctx->scratch.as<double>(), *T = M + nm;
  combine_jk<<<(int)std::min<size_t>((nm + 255) / 256, (size_t)num_sms() * 16), 256, 0, st>>>(J, K, cJ, cK, M, nm);
  dim3 thr(16, 16);
  // T[q] = M[q] C_right            ([N][N] x [N][nr])
  gemm_f64<false><<<dim3((nr + 15) / 16, (N + 15) / 16, ndens), thr, 0, st>>>(
      M, (long long)N * N, C_right, 0, T, (long long)N * nr, N, nr, N, N, nr, nr);
  // F[q] = C_left^T T[q]           ([nl][N] x [N][nr])
  gemm_f64<false, true><<<dim3((nr + 15) / 16, (nl + 15) / 16, ndens), thr, 0, st>>>(
      C_left, 0, T, (long long)N * nr, F, (long long)nl * nr, nl, nr, N, nl, nr, nr);
  CUDA_TRY(cudaGetLastError());
  g_launches += 3;
  return LTJK_OK;
}

int ltjk_shell_quartets(ltjk_ctx *ctx, int nq, const int *shells_host, int precision, double *out,
                        ltjk_stream stream) {
  if (!ctx || !shells_host || !out || nq < 0) return set_error(LTJK_EINVAL, "shell_quartets: bad argument");
  if (precision != LTJK_FP64 && precision != LTJK_MIXED && precision != LTJK_FP64_NATIVE)
    return set_error(LTJK_EINVAL, "shell_quartets: bad precision");
  CUDA_TRY(cudaSetDevice(ctx->device));
  std::vector<std::pair<int, int>> qs;
  for (int k = 0; k < nq; ++k) {
    const int *s = shells_host + 4 * k;
    for (int t = 0; t < 4; ++t)
      if (s[t] < 0 || s[t] >= ctx->nshells) return set_error(LTJK_EINVAL, "shell_quartets: shell index");
    auto i = ctx->pair_of.find({s[0], s[1]}), j = ctx->pair_of.find({s[2], s[3]});
    if (i == ctx->pair_of.end() || j == ctx->pair_of.end())
      return set_error(LTJK_EINVAL,
                       "shell_quartets: pair (%d,%d) or (%d,%d) not in canonical order "
                       "(l_a > l_b, or l_a == l_b and a >= b)",
                       s[0], s[1], s[2], s[3]);
    qs.push_back({i->second, j->second});
  }
  std::vector<long long> offs;
  return store_blocks(*ctx, qs, precision, offs, out, reinterpret_cast<cudaStream_t>(stream));
}

int ltjk_alu_peak(int kind, double *flops, ltjk_stream stream) {
  if (!flops || kind < 0 || kind > 3) return set_error(LTJK_EINVAL, "alu_peak: kind must be 0..3");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = num_sms() * 4, threads = 256;
  const int iters = kind == 0 ? 16384 : kind == 1 ? 256 : 2048;
  switch (kind) {
    case 0: alu_peak_kernel<0><<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-3f); break;
    case 1: alu_peak_kernel<1><<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-3f); break;
    case 2: alu_peak_kernel<2><<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-3f); break;
    default: alu_peak_kernel<3><<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-3f); break;
  }
  CUDA_TRY(cudaGetLastError());
  g_launches += 1;
  *flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  return LTJK_OK;
}

int ltjk_class_program(int la, int lb, int lc, int ld, int deriv, ltjk_program_info *out) {
  if (!out) return set_error(LTJK_EINVAL, "class_program: null argument");
  if (deriv != 0 && deriv != 1) return set_error(LTJK_EINVAL, "class_program: deriv must be 0 or 1");
  const int lmax = deriv ? kMaxLGrad : kMaxL;
  for (int l : {la, lb, lc, ld})
    if (l < 0 || l > lmax)
      return set_error(LTJK_EUNSUPPORTED, "class_program: l = %d outside 0..%d%s", l, lmax,
                       deriv ? " (derivative programs)" : "");
  const ProgramSet *ps;
  int rc = program_set(&ps);
  if (rc) return rc;
  // programs are stored for l_a >= l_b and l_c >= l_d
  if (la < lb) std::swap(la, lb);
  if (lc < ld) std::swap(lc, ld);
  const ClassProg &p = ps->progs[quartet_index(la, lb, lc, ld, deriv)];
  *out = ltjk_program_info{};
  out->ltot = p.ltot;
  out->vrr_levels = p.nvrr_level;
  out->vrr_steps = p.nvrr_level ? ps->levels[p.vrr_level0 + p.nvrr_level] - ps->levels[p.vrr_level0] : 0;
  out->vrr_slots = p.vrr_size;
  out->accumulators = p.acc_total;
  out->hrr_slots = p.hrr_size;
  out->tiles = p.ntile;
  for (int t = 0; t < p.ntile; ++t) {
    const TileProg &T = ps->tiles[p.tile_begin + t];
    out->outputs = std::max(out->outputs, T.nout);
    const int steps = ps->levels[T.hrr_level0 + T.nhrr_level] - ps->levels[T.hrr_level0];
    out->hrr_steps = std::max(out->hrr_steps, steps);
    out->hrr_levels = std::max(out->hrr_levels, T.nhrr_level);
  }
  out->vrr_flops = p.vrr_flops;
  out->hrr_flops = p.hrr_flops;
  out->smem_per_warp[0] = make_launch(p, sizeof(double)).smem_per_warp;
  out->smem_per_warp[1] = make_launch(p, sizeof(dflt)).smem_per_warp;
  out->smem_per_warp[2] = make_launch(p, sizeof(float)).smem_per_warp;
  return LTJK_OK;
}

}  // extern "C"

// ------------------------------------------------- allocation-free J/K build
// Scratch of ltjk_jk_build_noalloc: a file-scope device array, so the call
// itself never allocates.  Every device that loads this library holds it
// (64 MiB) until the process exits.  Host code must not pass the symbol
// itself to a kernel (on the host it names a stand-in, not device memory);
// the device address is looked up once per device with cudaGetSymbolAddress.
namespace {
constexpr size_t kNoallocDoubles = size_t(8) << 20;  // 64 MiB of FP64 scratch
__device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];
std::mutex g_noalloc_mu;
std::map<int, double *> g_noalloc_ptr;  // device -> address of g_noalloc_scratch

int noalloc_scratch(int device, double **out) {
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  auto it = g_noalloc_ptr.find(device);
  if (it != g_noalloc_ptr.end()) {
    *out = it->second;
    return LTJK_OK;
  }
  double *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return set_error(LTJK_ECUDA, "jk_build_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
  g_noalloc_ptr[device] = p;
  *out = p;
  return LTJK_OK;
}
}  // namespace

extern "C" int ltjk_jk_build_noalloc(ltjk_ctx *ctx, int ndens, const double *D, double *J,
                                     double *K, ltjk_stream stream) {
  if (!ctx || !D) return set_error(LTJK_EINVAL, "jk_build_noalloc: null context or density");
  if (ndens < 1 || ndens > 4096)
    return set_error(LTJK_EINVAL, "jk_build_noalloc: ndens %d not in 1..4096", ndens);
  if (!J && !K) return LTJK_OK;
  const size_t need = jk_scratch_bytes(ctx, ndens) / sizeof(double);  // 4 to 7 n + ndens doubles
  if (need > kNoallocDoubles)
    return set_error(LTJK_EINVAL,
                     "jk_build_noalloc: %d densities of %d AOs need %zu bytes of scratch, above the "
                     "fixed %zu-byte limit (use ltjk_jk_build)",
                     ndens, ctx->nao, need * sizeof(double), kNoallocDoubles * sizeof(double));
  CUDA_TRY(cudaSetDevice(ctx->device));
  double *base = nullptr;
  int rc = noalloc_scratch(ctx->device, &base);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents; the prologue clears the accumulators
  JKArgs a;
  if ((rc = jk_prologue(ctx, D, base, ndens, J != nullptr, K != nullptr, st, &a))) return rc;
  if ((rc = launch_classes<kJK>(ctx, a, st))) return rc;
  return jk_epilogue(ctx, a, J, K, st);
}

#include "cholesky.cuh"
#include "service.cuh"
