"""A priori error bound of the mixed-precision J/K build (test infrastructure).

Mixed mode evaluates a kept quartet (ab|cd) in binary32 when its Schwarz
product Q_ab Q_cd is at most the promotion threshold, and in FP64 class
otherwise; accumulation across quartets is binary64.  If every binary32
quartet satisfies |delta (mu nu|lam sig)| <= eps Q_ab Q_cd (eps covers the
recurrences and the binary32 products and partial sums of the digestion), the
triangle inequality over Eq. jkbuild gives, per AO element,

    |delta J_mn| <= eps sum_{c,d: binary32} Q_ab Q_cd sum_{l in c, s in d} |D_ls|
    |delta K_mn| <= eps sum_{c,d: binary32} Q_ac Q_bd sum_{l in c, s in d} |D_ls|

with m in shell a and n in shell b (K_mn = sum_ls (m l|n s) D_ls).  The bound
is evaluated per shell block from the oracle's Schwarz factors and is
independent of the integral kernels."""
import numpy as np

# Largest binary32 error of one quartet element relative to Q_ab Q_cd over the
# quartets mixed mode evaluates in binary32: the recurrences lose digits to
# cancellation on tight exponents (up to 5e3); the worst, (pp|pp), reaches
# 3.6e-3 on the 40-AO chain.  The margin covers the kernel's own rounding
# order (its stage-1 set-up in double-float, its primitive-group reduction).
EPS32 = 1e-2
# binary32 digestion: at most 100 products and partial sums per placement
# element (an f x f density block), plus the rounding of D: gamma_104 with
# u = 2^-24.
EPS_DIG = 104 * 2.0 ** -24
# A digestion of the binary32 quartets on tensor cores in TF32 (not built):
# each operand (integral, density) truncated to TF32's 10 explicit bits,
# relative error below u = 2^-10; the product of two TF32 values is exact in
# binary32 and the accumulation is binary32, so the operand rounding adds
# (1 + u)^2 - 1 = 2u + u^2 per product, and the binary32 sums stay within
# EPS_DIG as long as each accumulation chain has at most 100 terms.
EPS_TF32 = 2 * 2.0 ** -10 + 2.0 ** -20


def shell_block_abs(mol, D):
    """[ndens, ns, ns]: sum of |D_ls| over each shell block."""
    l = np.asarray(mol.shell_l)
    so = np.concatenate([[0], np.cumsum((l + 1) * (l + 2) // 2)])
    ns = len(l)
    A = np.abs(np.asarray(D))
    out = np.zeros((A.shape[0], ns, ns))
    for c in range(ns):
        for d in range(ns):
            out[:, c, d] = A[:, so[c]:so[c + 1], so[d]:so[d + 1]].sum(axis=(1, 2))
    return out


def mixed_jk_bound(Q, mol, D, eps, tau, tmix):
    """Largest bound on |delta J| and |delta K| over all elements and densities.

    Q: [ns, ns] Schwarz factors; tau: screening threshold (quartets with
    Q_ab Q_cd < tau are dropped, on both sides); tmix: promotion threshold.
    The binary32 set is taken with a relative margin of 1e-9 on tmix so that
    a quartet at the threshold counts as binary32 whichever way the two
    Schwarz computations round it."""
    Ds = shell_block_abs(mol, D)
    ns = Q.shape[0]
    bj = np.zeros((Ds.shape[0], ns, ns))
    bk = np.zeros((Ds.shape[0], ns, ns))
    for a in range(ns):
        # J: quartets (a b | c d), weight Q_ab Q_cd
        qq = Q[a][:, None, None] * Q[None, :, :]                       # [b, c, d]
        w = np.where((qq >= tau * (1 - 1e-9)) & (qq <= tmix * (1 + 1e-9)), qq, 0.0)
        bj[:, a, :] = np.einsum("bcd,ncd->nb", w, Ds)
        # K: quartets (a c | b d), weight Q_ac Q_bd
        qq = Q[a][:, None, None] * Q[None, :, :]                       # [c, b, d]
        w = np.where((qq >= tau * (1 - 1e-9)) & (qq <= tmix * (1 + 1e-9)), qq, 0.0)
        bk[:, a, :] = np.einsum("cbd,ncd->nb", w, Ds)
    return eps * bj.max(), eps * bk.max()
