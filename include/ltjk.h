/*
 * ltjk.h -- C ABI of the GB300 Laplace-transform AO-direct J/K library.
 *
 * The library computes, on one GPU, the Coulomb and exchange builds of many
 * non-symmetric AO densities with electron-repulsion integrals evaluated on the
 * fly over Schwarz-screened Cartesian Gaussian shell quartets, the Laplace
 * pseudo-densities that feed them, and the nuclear-gradient adjoint of the
 * build.  Equations are cited by the paper's labels (arXiv 2607.05622).
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: LTJK_OK (0) or a negative code
 *     below.  On failure ltjk_last_error() (thread-local) describes the cause
 *     and no output is guaranteed to be written.
 *   - Arrays are DEVICE pointers unless the argument name ends in _host.  The
 *     caller owns every array; the library never frees caller memory.
 *   - Matrices are row-major FP64.  A stack of n AO matrices is [n][N][N] with
 *     N = number of Cartesian AOs; element (q, mu, nu) sits at q*N*N + mu*N + nu.
 *   - AO order: shells in input order; within a shell of angular momentum l the
 *     Cartesian components x^lx y^ly z^lz ordered by descending lx, then
 *     descending ly.  A contracted shell is sum_k c_k N_k g_k with g_k the
 *     primitive of exponent a_k, N_k = (2a_k/pi)^{3/4} (4a_k)^{l/2} / sqrt((2l-1)!!)
 *     (unit norm for the x^l component), and the contracted x^l function is
 *     rescaled to unit self-overlap; other components are not rescaled.
 *   - Device work is enqueued on the caller's stream (a cudaStream_t passed as
 *     ltjk_stream; NULL = legacy default stream) and the call returns without
 *     waiting unless stated otherwise.  Input arrays must stay valid and
 *     unmodified, and outputs must not be read, until the stream reaches the
 *     point of the call.
 *   - A context is not thread-safe: calls on one context from several host
 *     threads must be serialised by the caller.  Distinct contexts are
 *     independent.
 */
#ifndef LTJK_H
#define LTJK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define LTJK_OK 0
#define LTJK_EINVAL (-1)        /* invalid argument (null pointer, bad size, bad basis) */
#define LTJK_ENOMEM (-2)        /* device or host allocation failed */
#define LTJK_EBUDGET (-3)       /* request does not fit the service's HBM budget */
#define LTJK_EUNSUPPORTED (-4)  /* angular momentum above the compiled maximum of the call */
#define LTJK_ECUDA (-5)         /* a CUDA runtime call failed */
#define LTJK_ETIMEDOUT (-6)     /* a bounded wait ran out */
#define LTJK_ECANCELLED (-7)    /* the request was cancelled */
#define LTJK_ENOTREADY (-8)     /* result not yet available */

#define LTJK_MAX_L 3            /* largest shell angular momentum of the J/K build (s, p, d, f) */
#define LTJK_MAX_L_GRAD 2       /* largest shell angular momentum of the gradient adjoint */
#define LTJK_MAX_PRIM 8         /* largest number of primitives in one shell */

#define LTJK_FP64 0         /* FP64-class: double-float recurrences and digestion */
#define LTJK_MIXED 1        /* FP32 below the Schwarz threshold, FP64-class above */
#define LTJK_FP64_NATIVE 2  /* every recurrence and digestion step in IEEE binary64 */

typedef struct CUstream_st *ltjk_stream;

/* Thread-local description of the last failure on this host thread. */
const char *ltjk_last_error(void);

/* Library version, MAJOR*10000 + MINOR*100 + PATCH. */
int ltjk_version(void);

/* Number of CUDA kernels this library has launched in this process (all
   devices, all contexts), for accounting.  Host-only. */
int ltjk_launch_count(unsigned long long *count);

/* --------------------------------------------------------------- contexts */
/* A molecule in a Cartesian contracted Gaussian basis.  All arrays are host
   arrays and are copied by ltjk_context_create.
     natoms, coords_host[natoms*3]      atom positions, bohr
     nshells                            number of shells
     shell_atom_host[nshells]           atom index of each shell (0..natoms-1)
     shell_l_host[nshells]              angular momentum, 0..LTJK_MAX_L
     shell_nprim_host[nshells]          number of primitives, 1..8
     exps_host[sum nprim]               primitive exponents (> 0), shell by shell
     coefs_host[sum nprim]              contraction coefficients with respect to
                                        unit-normalised primitives (see above) */
typedef struct {
  int natoms;
  const double *coords_host;
  int nshells;
  const int *shell_atom_host;
  const int *shell_l_host;
  const int *shell_nprim_host;
  const double *exps_host;
  const double *coefs_host;
} ltjk_basis;

/* Build options.
     schwarz_tau  shell quartet (ab|cd) is skipped iff Q_ab * Q_cd < schwarz_tau,
                  Q_ab = max over mu in a, nu in b of sqrt|(mu nu|mu nu)|
                  (plain Schwarz bound, not density weighted).  0 keeps all.
     mixed_tau    precision == LTJK_MIXED only: quartets with Q_ab*Q_cd > mixed_tau
                  are evaluated FP64-class, the rest in FP32 (Boys function always
                  FP64; J/K always accumulated in FP64).
     precision    LTJK_FP64, LTJK_MIXED or LTJK_FP64_NATIVE.  LTJK_FP64 (FP64
                  class) runs the Boys function, the per-primitive set-up, the
                  recurrences and the density digestion in double-float
                  arithmetic (pairs of FP32 words, about 2^-44 relative per
                  operation) on the FP32 pipe, which on GB300 is 58x faster
                  than its FP64 pipe; LTJK_FP64_NATIVE keeps every step in IEEE
                  binary64.  Both meet the FP64 parity gate (1e-10 relative to
                  the oracle).  In LTJK_FP64 (and the promoted quartets of
                  LTJK_MIXED) the classes with an f shell run in IEEE binary64:
                  their recurrences amplify rounding ~1e4-fold, too much for
                  double-float's ~2^-44 at that gate.  LTJK_MIXED evaluates
                  the quartets above mixed_tau as LTJK_FP64 and the rest with
                  binary32 recurrences and digestion (their Boys function and
                  set-up in double-float, rounded to binary32).  The accumulation across
                  quartets is IEEE binary64 in every mode.
                  Range: each density is scaled by the exact power of two that
                  brings its largest element into [1/2, 1) before the
                  double-float and binary32 copies are made, and J and K are
                  scaled back exactly, so D may take any binary64 magnitude
                  (elements below 2^-126 of their density's largest element
                  are flushed in the binary32 words of the FP64-class and
                  mixed modes: an absolute error far below their 1e-10 and
                  stated tolerances).
     device       CUDA device ordinal the context lives on. */
typedef struct {
  double schwarz_tau;
  double mixed_tau;
  int precision;
  int device;
} ltjk_opts;

typedef struct ltjk_ctx ltjk_ctx;

/* Work counts of a context (host values). */
typedef struct {
  int nao;
  int nshells;
  int npairs;                 /* shell pairs a >= b */
  int64_t quartets_total;     /* unique shell quartets before screening */
  int64_t quartets_kept;      /* unique shell quartets kept by Schwarz */
  int64_t quartets_fp64;      /* of those, evaluated in FP64 */
  int64_t prim_quartets_kept; /* primitive quartets over the kept shell quartets */
  int64_t cart_integrals_kept;/* contracted Cartesian integrals over the kept quartets */
  double eri_flops_per_build; /* recurrence flop model over the kept quartets */
  size_t device_bytes;        /* device memory held by the context */
  double eri_flops_fp64;      /* part of eri_flops_per_build in FP64-class quartets */
  int64_t cart_integrals_fp64;/* part of cart_integrals_kept in FP64-class quartets */
  double grad_eri_flops;      /* derivative-recurrence flop model over the kept quartets */
  double grad_eri_flops_fp64; /* part of grad_eri_flops in FP64-class quartets */
} ltjk_ctx_stats;

/* Create a context: normalises the basis, builds every shell pair and its
   primitive-pair data, evaluates the Schwarz factors on the device, sorts the
   pairs by class and Q and builds the screened quartet work lists (Schwarz
   screening, cf. the paper's Sect. "Cost" and its screening discussion).
   Synchronous.  *out receives the context (null on any error).  The basis and
   options are checked on the host before the first CUDA call: l above
   LTJK_MAX_L gives LTJK_EUNSUPPORTED; a negative l, a primitive count outside
   1..LTJK_MAX_PRIM, an atom index out of range, a non-positive or non-finite
   exponent, a non-finite coordinate, an unknown precision or a negative or
   NaN threshold give LTJK_EINVAL. */
int ltjk_context_create(const ltjk_basis *basis, const ltjk_opts *opts, ltjk_ctx **out);
/* Release a context.  Work that uses it must have completed: synchronise the
   streams it was used on (or wait for its service requests) first.  Device
   memory of the library is stream-ordered (cudaMallocAsync/cudaFreeAsync), so
   creating and destroying contexts never synchronises the whole device. */
int ltjk_context_destroy(ltjk_ctx *ctx);
int ltjk_nao(const ltjk_ctx *ctx, int *nao);
int ltjk_context_stats(const ltjk_ctx *ctx, ltjk_ctx_stats *out);

/* Schwarz factors of every ordered shell pair, Q_host[a*nshells + b]. Synchronous. */
int ltjk_schwarz(const ltjk_ctx *ctx, double *Q_host);

/* ------------------------------------------------------ Laplace quadrature */
/* Least-squares exponential sum sum_q w_q exp(-t_q x) ~ 1/x on [xmin, xmax]
   (Eq. laplace), fitted on the relative residual: the weights are the linear
   least-squares solution for given exponents (variable projection) and
   Levenberg-Marquardt moves the exponents, with continuation in the number
   of points.  Once an added point no longer lowers the residual (the fit has
   reached what double precision allows on the range), the remaining points
   are placed in the widest gaps with a weight of 1e-16 of the smallest, so
   n points are always returned.  The fit is made on [1, R_g] in units of
   xmin, log R_g = log(xmax / xmin) rounded up to a multiple of 1/8, so the
   nodes depend only on n and that cell (never on earlier calls); the steps
   of each continuation are cached per cell.  Host-only, synchronous,
   thread-safe.
     0 < xmin < xmax, 1 <= n <= 32; t_host[n], w_host[n] receive the nodes
     (strictly ascending) and weights (positive); *max_rel_err (nullable)
     receives max |x sum w exp(-t x) - 1| on 10^5 log-spaced points of
     [xmin, xmax]. */
int ltjk_laplace_quadrature(double xmin, double xmax, int n, double *t_host, double *w_host,
                            double *max_rel_err);

/* Minimax (best uniform relative error) exponential sum for 1/x on
   [xmin, xmax] -- the grid the paper prescribes (Eq. laplace): Lawson
   reweighting of the least-squares fit, then the Remez exchange (the
   levelled-error equations solved with the weights projected out); the
   relative error of the result equioscillates at 2n+1 points.  Host-only,
   synchronous.  Arguments as ltjk_laplace_quadrature; *converged (nullable)
   is 1 when the exchange levelled the error, 0 when it did not (the nodes
   returned are then the least-squares ones). */
int ltjk_laplace_minimax(double xmin, double xmax, int n, double *t_host, double *w_host,
                         double *max_rel_err, int *converged);

/* EOM excitation-energy shift of a grid (Eq. eomshift):
   w_shifted[q] = w[q] exp(omega t[q]), so that sum_q w_shifted[q] exp(-t[q] D)
   approximates 1/(D - omega) with the grid's relative accuracy wherever
   D - omega lies in the fitted range (valid for omega below the smallest
   denominator).  Host-only. */
int ltjk_laplace_shift(int n, const double *t_host, const double *w_host, double omega,
                       double *w_shifted_host);

/* --------------------------------------------------------- pseudo-densities */
/* D[q*npair + p] = U_q X_p V_q^T, U_q = C_occ diag(exp(+t_q eps_occ)),
   V_q = C_vir diag(exp(-t_q eps_vir)) (Eq. scaledcoeff; Eq. aodensk with the
   residual replaced by the transition amplitudes X_p).  No quadrature weight is
   applied.
     C_occ [N][nocc], C_vir [N][nvir], eps_occ [nocc], eps_vir [nvir] (device),
     X [npair][nocc][nvir] (device), t_host [nlap] (host),
     D [nlap*npair][N][N] (device, overwritten).  nocc, nvir, npair, nlap >= 1
     and npair * nlap <= 4096, else LTJK_EINVAL. */
int ltjk_pseudo_densities(ltjk_ctx *ctx, int nocc, int nvir, const double *C_occ,
                          const double *C_vir, const double *eps_occ, const double *eps_vir,
                          int npair, const double *X, int nlap, const double *t_host, double *D,
                          ltjk_stream stream);

/* ------------------------------------------------------------- J/K build */
/* J[q]_{mu nu} = sum_{ka rho} (mu nu|ka rho) D[q]_{ka rho},
   K[q]_{mu nu} = sum_{ka rho} (mu ka|nu rho) D[q]_{ka rho}   (Eq. jkbuild)
   for ndens arbitrary (non-symmetric) D[q], over the Schwarz-kept quartets,
   ERIs recomputed on the fly in the context's precision.
     D [ndens][N][N] in; J, K [ndens][N][N] out (overwritten; either may be
     NULL to skip it).  1 <= ndens <= 4096.  Uses internal device scratch
     (held by the context, grown on demand). */
int ltjk_jk_build(ltjk_ctx *ctx, int ndens, const double *D, double *J, double *K,
                  ltjk_stream stream);

/* The same build as ltjk_jk_build, but the call allocates no device memory:
   its scratch is a fixed 64 MiB array inside the library (held by every GPU
   that loads the library until the process exits).  This is for callers that
   cannot let a library allocate: applications that own all device memory
   through their own pool or framework allocator, or latency-critical loops
   that cannot absorb the device-wide synchronisation of cudaMalloc/cudaFree.
   The paper has no counterpart; this is an interface convenience.
     Limit: 4 * ndens * N * N + ndens doubles (FP64 contexts) or
     5 * ndens * N * N + ndens (mixed contexts), two more ndens * N * N for
     an FP64-class or mixed context with an f shell (binary64 density copies
     beside the double-float ones), must not exceed 8 * 2^20;
     larger requests return LTJK_EINVAL with the sizes in ltjk_last_error().
     The first call on each device looks up the array's device address
     (cudaGetSymbolAddress) with that device current; make that first call
     before any stream capture.
     All calls share the one array and it keeps the previous call's contents
     (the accumulators are cleared on every call): calls that can overlap on
     the GPU (different streams, or different host threads) race and give
     wrong results; serialise them.
   Arguments, layouts and results are those of ltjk_jk_build. */
int ltjk_jk_build_noalloc(ltjk_ctx *ctx, int ndens, const double *D, double *J, double *K,
                          ltjk_stream stream);

/* F[q] = cJ J[D_q] + cK K[D_q]: the combination a gradient's adjoint with
   respect to a density takes (Eq. jkderiv: dE/dP_r = cJ J[Q_r] + cK K[Q_r]
   for E = sum_r [cJ J(P_r, Q_r) + cK K(P_r, Q_r)]), formed in the build's
   epilogue.  D, F [ndens][N][N] device (F overwritten; D and F must not
   overlap); 1 <= ndens <= 4096; a zero coefficient skips that build.  Uses
   the context's scratch. */
int ltjk_jk_fock(ltjk_ctx *ctx, int ndens, const double *D, double cJ, double cK, double *F,
                 ltjk_stream stream);

/* The energy functional of the gradient adjoint,
     E = sum_r <P_r, cJ J[Q_r] + cK K[Q_r]> = sum_r [cJ J(P_r, Q_r) + cK K(P_r, Q_r)]
   (Eq. jkderiv; <A, B> = sum_{mu nu} A_{mu nu} B_{mu nu}), with F = cJ J[Q] +
   cK K[Q] from ltjk_jk_fock.  P, Q [nterms][N][N] device; F [nterms][N][N]
   device (written, nullable: then kept in scratch); E one device double
   (overwritten).  The sum over elements is taken in a fixed order (no
   atomics); F itself carries the build's atomic accumulation order, so two
   calls agree to rounding.  1 <= nterms <= 4096. */
int ltjk_jk_energy(ltjk_ctx *ctx, int nterms, const double *P, const double *Q, double cJ,
                   double cK, double *F, double *E, ltjk_stream stream);

/* ---------------------------------------------------------- gradient adjoint */
/* grad[A][x] = d/dR_{A,x} sum_r [cJ J(P_r, Q_r) + cK K(P_r, Q_r)] with the
   ordered builds J(A,B) = sum (mu nu|ka rho) A_{mu nu} B_{ka rho} and
   K(A,B) = sum (mu ka|nu rho) A_{mu nu} B_{ka rho} (Eq. jkderiv); derivative
   integrals for three centres, the fourth by translational invariance
   (Eq. l18).  Only the two-electron term: no one-electron or nuclear part.
     P, Q [nterms][N][N] (device, any symmetry), grad [natoms][3] (device,
     overwritten).  1 <= nterms <= 4096.  Shells up to LTJK_MAX_L_GRAD (d):
     a context with an f shell gives LTJK_EUNSUPPORTED before any launch (the
     derivative programs of f quartets need one more unit, g, and their
     contracted accumulators alone, 29340 of them for (ff|ff), exceed a
     warp's shared memory). */
int ltjk_jk_grad(ltjk_ctx *ctx, int nterms, const double *P, const double *Q, double cJ,
                 double cK, double *grad, ltjk_stream stream);

/* ----------------------------------------------- Laplace-Fock back-transform */
/* F[q] = C_left^T (cJ J[q] + cK K[q]) C_right (Eq. laplacefock with cJ = 2,
   cK = -1 and C_left = C_right = C): returns each grid point's J/K build to the
   MO basis; with C_left = C_occ and C_right = C_vir it gives the
   occupied-virtual block that feeds the next level of the density cascade
   (Eq. aodensk, through ltjk_pseudo_densities with X = that block).
     J, K [ndens][N][N], C_left [N][nl], C_right [N][nr] (device, row-major),
     F [ndens][nl][nr] (device, overwritten).  Uses the context's scratch. */
int ltjk_laplace_fock(ltjk_ctx *ctx, int ndens, const double *J, const double *K, double cJ,
                      double cK, int nl, const double *C_left, int nr, const double *C_right,
                      double *F, ltjk_stream stream);

/* ------------------------------------------------------- measurement */
/* One launch of an arithmetic-throughput kernel on the caller's stream (the
   roofline denominators of the benchmark; not part of the method): every
   thread of a grid of 4 CTAs x 256 threads per SM runs 8 independent chains of
   fused multiply-adds.  kind 0: binary32 FMA; 1: binary64 FMA; 2: double-float
   FMA (the FP64-class arithmetic of the recurrences); 3: the double-float
   dot-product accumulation of the density digestion.  *flops (host) receives
   the algorithmic flops of one launch (2 per multiply-add); time the launch
   with events on the stream.  The kernel's results go to a file-scope device
   word (nothing is allocated). */
int ltjk_alu_peak(int kind, double *flops, ltjk_stream stream);

/* ------------------------------------------------------ spherical AOs */
/* Matrix-level Cartesian <-> real-spherical transformation.  The paper works
   in Cartesian shells (Computational Details); this maps AO matrices to real
   spherical functions, T block diagonal over the shells: s 1; p x, y, z (the
   Cartesian order); d, m = -2..2: sqrt3 xy, sqrt3 yz, (2 zz - xx - yy)/2,
   sqrt3 xz, sqrt3 (xx - yy)/2; f, m = -3..3: sqrt(5/8) y(3xx - yy),
   sqrt15 xyz, sqrt(3/8) y(4zz - xx - yy), z(2zz - 3xx - 3yy)/2,
   sqrt(3/8) x(4zz - xx - yy), sqrt15/2 z(xx - yy), sqrt(5/8) x(xx - 3yy);
   with every Cartesian component normalised as x^l.  direction 0: B[q] = T A[q] T^T (A [ndens][N][N] Cartesian, e.g. J
   or K, to B [ndens][Ns][Ns]); direction 1: B[q] = T^T A[q] T (a spherical
   density A [ndens][Ns][Ns] to the Cartesian B [ndens][N][N] the build
   takes).  IEEE FP64, device arrays; uses the context's scratch.
   ltjk_nsph gives Ns = sum over shells of 2l+1. */
int ltjk_nsph(const ltjk_ctx *ctx, int *nsph);
int ltjk_sph_transform(ltjk_ctx *ctx, int direction, int ndens, const double *A, double *B,
                       ltjk_stream stream);

/* ----------------------------------------------- Cholesky-factorised J/K */
/* Pivoted incomplete Cholesky factor of the ERI matrix over AO pairs
   (Eq. cdfact): (mu nu|ka rho) ~ sum_Q B[Q][mu][nu] B[Q][ka][rho].  Starting
   from the residual diagonal (mu nu|mu nu), it repeatedly takes the unique
   pair mu >= nu with the largest residual diagonal (lowest index on ties)
   while that exceeds delta, evaluates the ERI columns of the pivot's shell
   pair with the direct build's quartet kernels (IEEE FP64, cached for later
   pivots of the same pair) and appends the vector
   (V[:, p] - sum_Q B[Q] B[Q][p]) / sqrt(d_p).  Synchronous.
     delta > 0, max_vectors >= 1; B [max_vectors][N][N] device, caller-owned
     (row Q is a symmetric matrix; rows >= *naux are left untouched);
     *naux receives the number of vectors, *max_residual (nullable) the
     largest residual diagonal left, which bounds every element of
     V - B^T B (the residual is positive semidefinite).  The factorisation
     stops at max_vectors even if the residual is still above delta. */
int ltjk_cd_factor(ltjk_ctx *ctx, double delta, int max_vectors, double *B, int *naux,
                   double *max_residual, ltjk_stream stream);

/* J and K of densities given as factors, D[q] = U[q] V[q]^T, read off the
   Cholesky factor (Eq. cdj: J = sum_Q B_Q gamma_Q, gamma_Q = <B_Q, D>;
   Eq. cdknonsym: K = sum_{Q,m} (B_Q U)_{mu m} (B_Q V)_{nu m}).  A Laplace
   pseudo-density D_q = C_occ Y_q C_vir^T has rank nocc with one left factor
   for all densities: U = C_occ (u_count = 1), V_q = C_vir Y_q^T; a general D
   is U = D, V = identity (rank N, u_count = ndens).
   Precision follows the context: IEEE FP64 for LTJK_FP64_NATIVE; otherwise
   the products B U, B V and sum_Q (B_Q U)(B_Q V)^T run as double-float GEMMs
   on the FP32 pipe (~2^-44 relative per operation, FP64 accumulation of the
   split-k partial sums) and J's final contraction in IEEE FP64.
     B [naux][N][N] from ltjk_cd_factor; U [u_count][N][rank] and
     V [ndens][N][rank] device, row-major, u_count 1 or ndens; J, K
     [ndens][N][N] device, overwritten (either may be NULL).
     1 <= ndens <= 4096, 1 <= rank <= N.  Uses the context's scratch (up to
     about 2 GB of density chunks plus the left-factor products). */
int ltjk_cd_jk(ltjk_ctx *ctx, int naux, const double *B, int ndens, int rank, int u_count,
               const double *U, const double *V, double *J, double *K, ltjk_stream stream);

/* The Laplace pseudo-densities of ltjk_pseudo_densities as rank-nocc factors,
   D[q*npair + p] = U[q*npair + p] V[q*npair + p]^T with U = C_occ and
   V = C_vir Y^T, Y = exp(t_q (eps_i - eps_a)) X_p (Eq. scaledcoeff): the
   input of ltjk_cd_jk.  Arguments as ltjk_pseudo_densities; U, V
   [nlap*npair][N][nocc] device, overwritten.  Uses the context's scratch. */
int ltjk_pseudo_density_factors(ltjk_ctx *ctx, int nocc, int nvir, const double *C_occ,
                                const double *C_vir, const double *eps_occ, const double *eps_vir,
                                int npair, const double *X, int nlap, const double *t_host, double *U,
                                double *V, ltjk_stream stream);

/* ------------------------------------------------------------- inspection */
/* Contracted Cartesian integral blocks of nq shell quartets (a,b|c,d) given in
   shells_host[4*nq]; out [sum of block sizes] device FP64, blocks concatenated
   in order, each [na][nb][nc][nd] row-major.  Evaluated by the same kernels as
   the build: double-float (LTJK_FP64; IEEE FP64 for classes with an f
   shell), FP32 (LTJK_MIXED) or IEEE FP64 (LTJK_FP64_NATIVE). */
int ltjk_shell_quartets(ltjk_ctx *ctx, int nq, const int *shells_host, int precision,
                        double *out, ltjk_stream stream);

/* The recurrence program of one shell-quartet class (the Obara-Saika vertical
   and Head-Gordon-Pople horizontal recurrences of the paper's "Computational
   Details", generated once per process): sizes and the flop model.  Generates
   and validates every program on first use (every slot in range, and no
   recurrence level writes a slot that the same level reads, so the lanes of a
   warp can run a level's steps in any order).  Host-only, no device needed.
     0 <= la, lb, lc, ld <= LTJK_MAX_L; deriv 0 (integrals) or 1 (derivative
     integrals, one extra unit of angular momentum; l up to LTJK_MAX_L_GRAD);
     *out is overwritten.  The integrals of the heavier value classes are
     produced in output tiles over the first index (a range of a's Cartesian
     components per tile), so that a tile's horizontal recurrence fits the
     warp's shared memory; derivative classes have nine tiles, one per
     (centre, direction).
   LTJK_EUNSUPPORTED for l above LTJK_MAX_L (LTJK_MAX_L_GRAD with deriv = 1),
   LTJK_EINVAL for a null out. */
typedef struct {
  int ltot;              /* la+lb+lc+ld (+1 for derivatives) */
  int vrr_steps, vrr_levels, vrr_slots;   /* vertical recurrence per primitive quartet */
  int accumulators;      /* contracted [e0|f0] values, all channels */
  int hrr_steps, hrr_levels, hrr_slots;   /* horizontal recurrence, largest output tile */
  int tiles, outputs;    /* output tiles; integrals of the largest tile (na nb nc nd
                            when the class has one value tile or is a derivative) */
  double vrr_flops;      /* flop model per primitive quartet (recurrence only) */
  double hrr_flops;      /* flop model per contracted quartet */
  size_t smem_per_warp[3]; /* bytes per warp: IEEE FP64, double-float, FP32 */
} ltjk_program_info;
int ltjk_class_program(int la, int lb, int lc, int ld, int deriv, ltjk_program_info *out);

/* --------------------------------------------------------------- serving */
/* A continuous-batching solver service on one device.  A scheduler thread
   admits submitted requests first-come-first-served whenever their device
   scratch fits the HBM budget (one slab allocated at creation, first-fit with
   adjacent-block coalescing), and advances every admitted request together in
   steps: each step launches, per quartet class, one kernel over the next chunk
   of work items of all active requests of that class, so requests that arrive
   while others run share the device.  Each request completes on its own; its
   result equals the stand-alone ltjk_jk_build / ltjk_jk_grad result up to the
   order of floating-point additions.  Contexts (resident shell-pair data) are
   owned by the caller and must outlive their requests; a context may serve
   several concurrent requests.  Inputs must be complete on the device when
   ltjk_service_submit is called; outputs are valid once ltjk_service_wait
   returns LTJK_OK (or poll reports done with LTJK_OK). */
typedef struct ltjk_service ltjk_service;

#define LTJK_REQ_JK 0
#define LTJK_REQ_GRAD 1

typedef struct {
  int kind;            /* LTJK_REQ_JK or LTJK_REQ_GRAD */
  ltjk_ctx *ctx;       /* molecule and precision (caller-owned) */
  int n;               /* densities (J/K) or terms (gradient), 1..4096 */
  const double *D;     /* J/K: [n][N][N] device, read */
  double *J, *K;       /* J/K: [n][N][N] device, written (either may be NULL) */
  const double *P, *Q; /* gradient: [n][N][N] device, read */
  double cJ, cK;       /* gradient coefficients (see ltjk_jk_grad) */
  double *grad;        /* gradient: [natoms][3] device, written */
} ltjk_request;

typedef struct {
  uint64_t submitted, completed, cancelled, failed;
  double p50_ms, p99_ms, mean_ms;  /* latency submit -> completion, completed requests */
  double throughput_rps;           /* completed / (last completion - first submission) */
  size_t bytes_in_use, bytes_peak, budget;
  uint64_t steps, launches;
  int active, queued;
} ltjk_svc_stats;

/* Create a service with an HBM budget (bytes, >= 1 MiB, allocated now) on a device. */
int ltjk_service_create(size_t hbm_budget_bytes, int device, ltjk_service **out);
/* Queue a request; *ticket identifies it.  LTJK_EBUDGET if it can never fit;
   LTJK_EUNSUPPORTED for a gradient request on a context with an f shell. */
int ltjk_service_submit(ltjk_service *svc, const ltjk_request *req, uint64_t *ticket);
/* Non-blocking: *done = 1 once finished; then returns the request's status. */
int ltjk_service_poll(ltjk_service *svc, uint64_t ticket, int *done);
/* Wait at most timeout_s seconds: LTJK_OK, LTJK_ETIMEDOUT (request continues),
   LTJK_ECANCELLED, or the request's failure code.  Never waits unboundedly. */
int ltjk_service_wait(ltjk_service *svc, uint64_t ticket, double timeout_s);
/* Cancel: a queued request is dropped; an active one stops issuing work and
   releases its memory once its launched work has drained. */
int ltjk_service_cancel(ltjk_service *svc, uint64_t ticket);
int ltjk_service_stats(ltjk_service *svc, ltjk_svc_stats *out);
/* Fault injection for tests: the next `count` admissions fail with LTJK_ENOMEM
   as if the allocation had failed; other requests are unaffected. */
int ltjk_service_fail_next_admission(ltjk_service *svc, int count);
/* Cancel queued requests, drain active ones, stop the scheduler, free the slab. */
int ltjk_service_destroy(ltjk_service *svc);

#ifdef __cplusplus
}
#endif
#endif /* LTJK_H */
