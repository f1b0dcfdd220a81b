"""Python binding of the C ABI in include/ltjk.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/libltjk.so``; PyTorch is
used for device memory and streams.  There is no fallback: if the library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libltjk.so")

OK, EINVAL, ENOMEM, EBUDGET, EUNSUPPORTED, ECUDA, ETIMEDOUT, ECANCELLED, ENOTREADY = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
FP64, MIXED, FP64_NATIVE = 0, 1, 2
MAX_L = 3          # largest shell l of the J/K build (f)
MAX_L_GRAD = 2     # largest shell l of the gradient adjoint (d)


class LtjkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ltjk error {code}: {msg}")
        self.code = code


class _Basis(ctypes.Structure):
    _fields_ = [("natoms", ctypes.c_int), ("coords_host", ctypes.c_void_p),
                ("nshells", ctypes.c_int), ("shell_atom_host", ctypes.c_void_p),
                ("shell_l_host", ctypes.c_void_p), ("shell_nprim_host", ctypes.c_void_p),
                ("exps_host", ctypes.c_void_p), ("coefs_host", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("schwarz_tau", ctypes.c_double), ("mixed_tau", ctypes.c_double),
                ("precision", ctypes.c_int), ("device", ctypes.c_int)]


class CtxStats(ctypes.Structure):
    _fields_ = [("nao", ctypes.c_int), ("nshells", ctypes.c_int), ("npairs", ctypes.c_int),
                ("quartets_total", ctypes.c_int64), ("quartets_kept", ctypes.c_int64),
                ("quartets_fp64", ctypes.c_int64), ("prim_quartets_kept", ctypes.c_int64),
                ("cart_integrals_kept", ctypes.c_int64), ("eri_flops_per_build", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("eri_flops_fp64", ctypes.c_double),
                ("cart_integrals_fp64", ctypes.c_int64), ("grad_eri_flops", ctypes.c_double),
                ("grad_eri_flops_fp64", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProgramInfo(ctypes.Structure):
    _fields_ = [("ltot", ctypes.c_int), ("vrr_steps", ctypes.c_int), ("vrr_levels", ctypes.c_int),
                ("vrr_slots", ctypes.c_int), ("accumulators", ctypes.c_int), ("hrr_steps", ctypes.c_int),
                ("hrr_levels", ctypes.c_int), ("hrr_slots", ctypes.c_int), ("tiles", ctypes.c_int),
                ("outputs", ctypes.c_int), ("vrr_flops", ctypes.c_double), ("hrr_flops", ctypes.c_double),
                ("smem_per_warp", ctypes.c_size_t * 3)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["smem_per_warp"] = list(self.smem_per_warp)
        return d


_lib = None

# exported symbols and their signatures (restype int unless noted)
_P, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "ltjk_last_error": ([], ctypes.c_char_p),
    "ltjk_version": ([], _I),
    "ltjk_launch_count": ([_P], _I),
    "ltjk_context_create": ([_P, _P, _P], _I),
    "ltjk_context_destroy": ([_P], _I),
    "ltjk_nao": ([_P, _P], _I),
    "ltjk_context_stats": ([_P, _P], _I),
    "ltjk_schwarz": ([_P, _P], _I),
    "ltjk_laplace_quadrature": ([_D, _D, _I, _P, _P, _P], _I),
    "ltjk_laplace_minimax": ([_D, _D, _I, _P, _P, _P, _P], _I),
    "ltjk_laplace_shift": ([_I, _P, _P, _D, _P], _I),
    "ltjk_pseudo_densities": ([_P, _I, _I, _P, _P, _P, _P, _I, _P, _I, _P, _P, _P], _I),
    "ltjk_jk_build": ([_P, _I, _P, _P, _P, _P], _I),
    "ltjk_jk_build_noalloc": ([_P, _I, _P, _P, _P, _P], _I),
    "ltjk_jk_grad": ([_P, _I, _P, _P, _D, _D, _P, _P], _I),
    "ltjk_jk_fock": ([_P, _I, _P, _D, _D, _P, _P], _I),
    "ltjk_alu_peak": ([_I, _P, _P], _I),
    "ltjk_jk_energy": ([_P, _I, _P, _P, _D, _D, _P, _P, _P], _I),
    "ltjk_shell_quartets": ([_P, _I, _P, _I, _P, _P], _I),
    "ltjk_class_program": ([_I, _I, _I, _I, _I, _P], _I),
    "ltjk_nsph": ([_P, _P], _I),
    "ltjk_sph_transform": ([_P, _I, _I, _P, _P, _P], _I),
    "ltjk_cd_factor": ([_P, ctypes.c_double, _I, _P, _P, _P, _P], _I),
    "ltjk_cd_jk": ([_P, _I, _P, _I, _I, _I, _P, _P, _P, _P, _P], _I),
    "ltjk_pseudo_density_factors": ([_P, _I, _I, _P, _P, _P, _P, _I, _P, _I, _P, _P, _P, _P], _I),
    "ltjk_laplace_fock": ([_P, _I, _P, _P, _D, _D, _I, _P, _I, _P, _P, _P], _I),
    "ltjk_service_create": ([ctypes.c_size_t, _I, _P], _I),
    "ltjk_service_submit": ([_P, _P, _P], _I),
    "ltjk_service_poll": ([_P, ctypes.c_uint64, _P], _I),
    "ltjk_service_wait": ([_P, ctypes.c_uint64, _D], _I),
    "ltjk_service_cancel": ([_P, ctypes.c_uint64], _I),
    "ltjk_service_stats": ([_P, _P], _I),
    "ltjk_service_fail_next_admission": ([_P, _I], _I),
    "ltjk_service_destroy": ([_P], _I),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} missing "
                               "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        msg = lib().ltjk_last_error()
        raise LtjkError(rc, msg.decode() if msg else "")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, shape=None, name="tensor", device=None):
    """Device pointer of a contiguous CUDA float64 tensor of the given shape, on
    GPU `device` when given (the library's kernels run on the context's GPU)."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise ValueError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the context is on cuda:{device}")
    return ctypes.c_void_p(t.data_ptr())


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    c = ctypes.c_ulonglong(0)
    _check(lib().ltjk_launch_count(ctypes.byref(c)))
    return c.value


ALU_FP32, ALU_FP64, ALU_DFLOAT_FMA, ALU_DFLOAT_DOT = 0, 1, 2, 3


def alu_peak(kind: int, stream=None) -> float:
    """ltjk_alu_peak: launch one arithmetic-throughput kernel on the stream;
    returns its algorithmic flops (time it with CUDA events)."""
    f = ctypes.c_double(0.0)
    _check(lib().ltjk_alu_peak(int(kind), ctypes.byref(f), _stream(stream)))
    return f.value


def class_program(la: int, lb: int, lc: int, ld: int, deriv: int = 0) -> dict:
    """ltjk_class_program: sizes and flop model of one class's recurrence program
    (host-only; generates and validates every program on first use)."""
    info = ProgramInfo()
    _check(lib().ltjk_class_program(la, lb, lc, ld, deriv, ctypes.byref(info)))
    return info.as_dict()


def laplace_quadrature(xmin: float, xmax: float, n: int):
    """(t, w, max_rel_err) of the least-squares exponential sum for 1/x (Eq. laplace)."""
    t = np.zeros(n)
    w = np.zeros(n)
    err = ctypes.c_double(0.0)
    _check(lib().ltjk_laplace_quadrature(float(xmin), float(xmax), int(n),
                                         t.ctypes.data_as(_P), w.ctypes.data_as(_P),
                                         ctypes.byref(err)))
    return t, w, err.value


def laplace_minimax(xmin: float, xmax: float, n: int):
    """(t, w, max_rel_err, converged) of the minimax exponential sum for 1/x (Eq. laplace)."""
    t = np.zeros(n)
    w = np.zeros(n)
    err = ctypes.c_double(0.0)
    conv = ctypes.c_int(0)
    _check(lib().ltjk_laplace_minimax(float(xmin), float(xmax), int(n), t.ctypes.data_as(_P),
                                      w.ctypes.data_as(_P), ctypes.byref(err), ctypes.byref(conv)))
    return t, w, err.value, bool(conv.value)


def laplace_shift(t, w, omega: float):
    """Shifted weights w exp(omega t) for 1/(D - omega) (Eq. eomshift)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    _check(lib().ltjk_laplace_shift(len(t), t.ctypes.data_as(_P), w.ctypes.data_as(_P),
                                    float(omega), out.ctypes.data_as(_P)))
    return out


class Context:
    """A molecule on the GPU: shell pairs, Schwarz factors and screened work lists."""

    def __init__(self, mol, schwarz_tau=1e-12, mixed_tau=1e-6, precision=FP64, device=0):
        self._keep = [np.ascontiguousarray(mol.coords, dtype=np.float64),
                      np.ascontiguousarray(mol.shell_atom, dtype=np.int32),
                      np.ascontiguousarray(mol.shell_l, dtype=np.int32),
                      np.ascontiguousarray(mol.shell_nprim, dtype=np.int32),
                      np.ascontiguousarray(mol.exps, dtype=np.float64),
                      np.ascontiguousarray(mol.coefs, dtype=np.float64)]
        c, a, l, n, e, k = self._keep
        b = _Basis(c.shape[0], c.ctypes.data, l.shape[0], a.ctypes.data, l.ctypes.data,
                   n.ctypes.data, e.ctypes.data, k.ctypes.data)
        o = _Opts(float(schwarz_tau), float(mixed_tau), int(precision), int(device))
        h = ctypes.c_void_p()
        torch.cuda.set_device(device)
        _check(lib().ltjk_context_create(ctypes.byref(b), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.device = device
        self.natoms = c.shape[0]
        self.nshells = l.shape[0]
        nao = ctypes.c_int()
        _check(lib().ltjk_nao(h, ctypes.byref(nao)))
        self.nao = nao.value
        self.precision = precision

    def close(self):
        if getattr(self, "_h", None):
            lib().ltjk_context_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = CtxStats()
        _check(lib().ltjk_context_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def schwarz(self) -> np.ndarray:
        Q = np.zeros((self.nshells, self.nshells))
        _check(lib().ltjk_schwarz(self._h, Q.ctypes.data_as(_P)))
        return Q

    def jk_build(self, D: torch.Tensor, J=None, K=None, want_j=True, want_k=True, stream=None):
        nd, N = D.shape[0], self.nao
        dp = _dev(D, (nd, N, N), "D", device=self.device)
        if want_j and J is None:
            J = torch.empty_like(D)
        if want_k and K is None:
            K = torch.empty_like(D)
        jp = _dev(J, (nd, N, N), "J", device=self.device) if want_j else None
        kp = _dev(K, (nd, N, N), "K", device=self.device) if want_k else None
        _check(lib().ltjk_jk_build(self._h, nd, dp, jp, kp, _stream(stream)))
        return J, K

    def jk_build_noalloc(self, D: torch.Tensor, J: torch.Tensor, K: torch.Tensor, stream=None):
        """ltjk_jk_build_noalloc: the same build with the library's fixed scratch array;
        the library allocates nothing (J and K are the caller's)."""
        nd, N = D.shape[0], self.nao
        _check(lib().ltjk_jk_build_noalloc(self._h, nd, _dev(D, (nd, N, N), "D", device=self.device),
                                           _dev(J, (nd, N, N), "J", device=self.device), _dev(K, (nd, N, N), "K", device=self.device),
                                           _stream(stream)))
        return J, K

    def jk_fock(self, D: torch.Tensor, cJ=1.0, cK=0.0, F=None, stream=None):
        """ltjk_jk_fock: F[q] = cJ J[D_q] + cK K[D_q]."""
        nd, N = D.shape[0], self.nao
        if F is None:
            F = torch.empty_like(D)
        _check(lib().ltjk_jk_fock(self._h, nd, _dev(D, (nd, N, N), "D", device=self.device), float(cJ),
                                  float(cK), _dev(F, (nd, N, N), "F", device=self.device), _stream(stream)))
        return F

    def jk_energy(self, P: torch.Tensor, Q: torch.Tensor, cJ=1.0, cK=0.0, F=None, stream=None):
        """ltjk_jk_energy: (E, F) with F = cJ J[Q] + cK K[Q] and E = sum_r <P_r, F_r>
        (E a 0-dimensional device tensor)."""
        nt, N = P.shape[0], self.nao
        if F is None:
            F = torch.empty_like(Q)
        E = torch.empty((), dtype=torch.float64, device=P.device)
        _check(lib().ltjk_jk_energy(self._h, nt, _dev(P, (nt, N, N), "P", device=self.device),
                                    _dev(Q, (nt, N, N), "Q", device=self.device), float(cJ), float(cK),
                                    _dev(F, (nt, N, N), "F", device=self.device),
                                    _dev(E, (), "E", device=self.device), _stream(stream)))
        return E, F

    def jk_grad(self, P: torch.Tensor, Q: torch.Tensor, cJ=1.0, cK=0.0, grad=None, stream=None):
        nt, N = P.shape[0], self.nao
        pp = _dev(P, (nt, N, N), "P", device=self.device)
        qp = _dev(Q, (nt, N, N), "Q", device=self.device)
        if grad is None:
            grad = torch.empty((self.natoms, 3), dtype=torch.float64, device=P.device)
        gp = _dev(grad, (self.natoms, 3), "grad", device=self.device)
        _check(lib().ltjk_jk_grad(self._h, nt, pp, qp, float(cJ), float(cK), gp, _stream(stream)))
        return grad

    def pseudo_densities(self, C_occ, C_vir, eps_occ, eps_vir, X, t, D=None, stream=None):
        N = self.nao
        no, nv = C_occ.shape[1], C_vir.shape[1]
        npair = X.shape[0]
        t = np.ascontiguousarray(t, dtype=np.float64)
        nlap = t.shape[0]
        if D is None:
            D = torch.empty((nlap * npair, N, N), dtype=torch.float64, device=C_occ.device)
        _check(lib().ltjk_pseudo_densities(
            self._h, no, nv, _dev(C_occ, (N, no), "C_occ", device=self.device), _dev(C_vir, (N, nv), "C_vir", device=self.device),
            _dev(eps_occ, (no,), "eps_occ", device=self.device), _dev(eps_vir, (nv,), "eps_vir", device=self.device), npair,
            _dev(X, (npair, no, nv), "X", device=self.device), nlap, t.ctypes.data_as(_P),
            _dev(D, (nlap * npair, N, N), "D", device=self.device), _stream(stream)))
        return D

    @property
    def nsph(self) -> int:
        n = ctypes.c_int()
        _check(lib().ltjk_nsph(self._h, ctypes.byref(n)))
        return n.value

    def to_spherical(self, A: torch.Tensor, stream=None):
        """ltjk_sph_transform direction 0: T A[q] T^T (Cartesian matrices to spherical)."""
        nd, N, Ns = A.shape[0], self.nao, self.nsph
        B = torch.empty((nd, Ns, Ns), dtype=torch.float64, device=A.device)
        _check(lib().ltjk_sph_transform(self._h, 0, nd, _dev(A, (nd, N, N), "A", device=self.device), _dev(B, name="B", device=self.device),
                                        _stream(stream)))
        return B

    def from_spherical(self, A: torch.Tensor, stream=None):
        """ltjk_sph_transform direction 1: T^T A[q] T (spherical densities to Cartesian)."""
        nd, N, Ns = A.shape[0], self.nao, self.nsph
        B = torch.empty((nd, N, N), dtype=torch.float64, device=A.device)
        _check(lib().ltjk_sph_transform(self._h, 1, nd, _dev(A, (nd, Ns, Ns), "A", device=self.device), _dev(B, name="B", device=self.device),
                                        _stream(stream)))
        return B

    def cd_factor(self, delta: float, max_vectors: int, stream=None):
        """ltjk_cd_factor (Eq. cdfact): (B [naux][N][N] view of a [max_vectors][N][N]
        buffer, naux, largest residual diagonal)."""
        N = self.nao
        buf = torch.empty((int(max_vectors), N, N), dtype=torch.float64, device=f"cuda:{self.device}")
        naux = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        _check(lib().ltjk_cd_factor(self._h, float(delta), int(max_vectors), _dev(buf, name="B", device=self.device),
                                    ctypes.byref(naux), ctypes.byref(res), _stream(stream)))
        return buf[: naux.value], naux.value, res.value

    def pseudo_density_factors(self, C_occ, C_vir, eps_occ, eps_vir, X, t, stream=None):
        """ltjk_pseudo_density_factors: (U, V) [nlap*npair][N][nocc] with D = U V^T."""
        N = self.nao
        no, nv = C_occ.shape[1], C_vir.shape[1]
        npair = X.shape[0]
        t = np.ascontiguousarray(t, dtype=np.float64)
        nq = t.shape[0] * npair
        U = torch.empty((nq, N, no), dtype=torch.float64, device=C_occ.device)
        V = torch.empty_like(U)
        _check(lib().ltjk_pseudo_density_factors(
            self._h, no, nv, _dev(C_occ, (N, no), "C_occ", device=self.device), _dev(C_vir, (N, nv), "C_vir", device=self.device),
            _dev(eps_occ, (no,), "eps_occ", device=self.device), _dev(eps_vir, (nv,), "eps_vir", device=self.device), npair,
            _dev(X, (npair, no, nv), "X", device=self.device), t.shape[0], t.ctypes.data_as(_P), _dev(U, name="U", device=self.device),
            _dev(V, name="V", device=self.device), _stream(stream)))
        return U, V

    def cd_jk(self, B: torch.Tensor, U: torch.Tensor, V: torch.Tensor, J=None, K=None, stream=None):
        """ltjk_cd_jk (Eqs. cdj, cdknonsym): J and K of D[q] = U[q] V[q]^T from the
        factor B; U may hold one left factor shared by every density ([1][N][rank])."""
        naux, N = B.shape[0], self.nao
        nd, _, rank = V.shape
        nu = U.shape[0]
        if J is None:
            J = torch.empty((nd, N, N), dtype=torch.float64, device=V.device)
        if K is None:
            K = torch.empty((nd, N, N), dtype=torch.float64, device=V.device)
        _check(lib().ltjk_cd_jk(self._h, naux, _dev(B, (naux, N, N), "B", device=self.device), nd, rank, nu,
                                _dev(U, (nu, N, rank), "U", device=self.device), _dev(V, (nd, N, rank), "V", device=self.device),
                                _dev(J, (nd, N, N), "J", device=self.device), _dev(K, (nd, N, N), "K", device=self.device), _stream(stream)))
        return J, K

    def laplace_fock(self, J, K, C_left, C_right, cJ=2.0, cK=-1.0, F=None, stream=None):
        """F[q] = C_left^T (cJ J[q] + cK K[q]) C_right (Eq. laplacefock)."""
        nd, N = J.shape[0], self.nao
        nl, nr = C_left.shape[1], C_right.shape[1]
        if F is None:
            F = torch.empty((nd, nl, nr), dtype=torch.float64, device=J.device)
        _check(lib().ltjk_laplace_fock(self._h, nd, _dev(J, (nd, N, N), "J", device=self.device), _dev(K, (nd, N, N), "K", device=self.device),
                                       float(cJ), float(cK), nl, _dev(C_left, (N, nl), "C_left", device=self.device), nr,
                                       _dev(C_right, (N, nr), "C_right", device=self.device), _dev(F, (nd, nl, nr), "F", device=self.device),
                                       _stream(stream)))
        return F

    def shell_quartets(self, quartets, precision=FP64, stream=None):
        """Contracted blocks of (a b|c d) for each (a,b,c,d) in canonical pair order."""
        q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
        sizes = []
        ls = self._keep[2]
        for a, b, c, d in q:
            sizes.append(int(np.prod([(int(ls[s]) + 1) * (int(ls[s]) + 2) // 2 for s in (a, b, c, d)])))
        out = torch.zeros(max(sum(sizes), 1), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(lib().ltjk_shell_quartets(self._h, q.shape[0], q.ctypes.data_as(_P), int(precision),
                                         _dev(out, None, "out", device=self.device), _stream(stream)))
        torch.cuda.current_stream().synchronize()
        res, off = [], 0
        host = out.cpu().numpy()
        for (a, b, c, d), n in zip(q, sizes):
            shp = [(int(ls[s]) + 1) * (int(ls[s]) + 2) // 2 for s in (a, b, c, d)]
            res.append(host[off:off + n].reshape(shp))
            off += n
        return res


class JKEnergy(torch.autograd.Function):
    """E = sum_r <P_r, cJ J[Q_r] + cK K[Q_r]> = sum_r [cJ J(P_r,Q_r) + cK K(P_r,Q_r)].

    forward(coords, P, Q, mol, cJ, cK, opts) builds a context at ``coords`` and
    evaluates E with ltjk_jk_energy; backward gives dE/dcoords from
    ltjk_jk_grad (Eq. jkderiv) and dE/dP_r = cJ J[Q_r] + cK K[Q_r] (kept from
    the forward pass), dE/dQ_r = cJ J[P_r] + cK K[P_r] from ltjk_jk_fock (the
    adjoint of a J/K build is a J/K build).  The binding only scales the
    library's results by the upstream gradient."""

    @staticmethod
    def forward(ctx_, coords, P, Q, mol, cJ=1.0, cK=0.0, opts=None):
        opts = dict(opts or {})
        m = mol.with_coords(coords.detach().cpu().numpy().astype(np.float64))
        c = Context(m, **opts)
        E, F = c.jk_energy(P.detach().contiguous(), Q.detach().contiguous(), cJ, cK)
        ctx_.save_for_backward(P, Q, F)
        ctx_.c = c
        ctx_.cJ, ctx_.cK = cJ, cK
        ctx_.coords_device = coords.device
        return E

    @staticmethod
    def backward(ctx_, gE):
        P, Q, F = ctx_.saved_tensors
        c = ctx_.c
        gc = gP = gQ = None
        if ctx_.needs_input_grad[0]:
            g = c.jk_grad(P.detach().contiguous(), Q.detach().contiguous(), ctx_.cJ, ctx_.cK)
            gc = (g * gE).to(ctx_.coords_device)
        if ctx_.needs_input_grad[1]:
            gP = F * gE
        if ctx_.needs_input_grad[2]:
            gQ = c.jk_fock(P.detach().contiguous(), ctx_.cJ, ctx_.cK) * gE
        return gc, gP, gQ, None, None, None, None


REQ_JK, REQ_GRAD = 0, 1


class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ctx", ctypes.c_void_p), ("n", ctypes.c_int),
                ("D", ctypes.c_void_p), ("J", ctypes.c_void_p), ("K", ctypes.c_void_p),
                ("P", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("cJ", ctypes.c_double),
                ("cK", ctypes.c_double), ("grad", ctypes.c_void_p)]


class ServiceStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("throughput_rps", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t),
                ("bytes_peak", ctypes.c_size_t), ("budget", ctypes.c_size_t),
                ("steps", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("active", ctypes.c_int), ("queued", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Service:
    """Continuous-batching J/K and gradient service (ltjk_service_* in include/ltjk.h).

    Tensors passed to submit_* must stay alive and unmodified until the request
    finishes; the binding keeps references until wait() returns."""

    def __init__(self, hbm_budget_bytes: int, device: int = 0):
        h = ctypes.c_void_p()
        torch.cuda.set_device(device)
        _check(lib().ltjk_service_create(int(hbm_budget_bytes), int(device), ctypes.byref(h)))
        self._h = h
        self.device = device
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().ltjk_service_destroy(self._h))
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _submit(self, req, keep):
        torch.cuda.current_stream().synchronize()  # inputs complete on the device
        t = ctypes.c_uint64()
        _check(lib().ltjk_service_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def submit_jk(self, ctx: Context, D, J=None, K=None):
        nd, N = D.shape[0], ctx.nao
        if J is None:
            J = torch.empty_like(D)
        if K is None:
            K = torch.empty_like(D)
        req = _Request(REQ_JK, ctx._h.value, nd, _dev(D, (nd, N, N), "D", device=ctx.device).value,
                       _dev(J, (nd, N, N), "J", device=ctx.device).value, _dev(K, (nd, N, N), "K", device=ctx.device).value,
                       None, None, 0.0, 0.0, None)
        return self._submit(req, (ctx, D, J, K)), J, K

    def submit_grad(self, ctx: Context, P, Q, cJ=1.0, cK=0.0, grad=None):
        nt, N = P.shape[0], ctx.nao
        if grad is None:
            grad = torch.empty((ctx.natoms, 3), dtype=torch.float64, device=P.device)
        req = _Request(REQ_GRAD, ctx._h.value, nt, None, None, None,
                       _dev(P, (nt, N, N), "P", device=ctx.device).value, _dev(Q, (nt, N, N), "Q", device=ctx.device).value,
                       float(cJ), float(cK), _dev(grad, (ctx.natoms, 3), "grad", device=ctx.device).value)
        return self._submit(req, (ctx, P, Q, grad)), grad

    def poll(self, ticket):
        done = ctypes.c_int(0)
        rc = lib().ltjk_service_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(done))
        if done.value:
            self._keep.pop(ticket, None)
        return bool(done.value), rc

    def wait(self, ticket, timeout_s=60.0):
        rc = lib().ltjk_service_wait(self._h, ctypes.c_uint64(ticket), float(timeout_s))
        if rc != ETIMEDOUT:
            self._keep.pop(ticket, None)
        _check(rc)

    def cancel(self, ticket):
        _check(lib().ltjk_service_cancel(self._h, ctypes.c_uint64(ticket)))

    def fail_next_admission(self, count=1):
        _check(lib().ltjk_service_fail_next_admission(self._h, int(count)))

    def stats(self) -> dict:
        s = ServiceStats()
        _check(lib().ltjk_service_stats(self._h, ctypes.byref(s)))
        return s.as_dict()
