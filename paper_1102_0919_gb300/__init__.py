"""Python binding of the GB300 self-learning AMG triplet solver (C ABI in
include/samg.h).  Argument marshalling only: every step of the setup and
solve phases runs in the library's CUDA kernels (and its host C++ setup
code).  Importing this package fails if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsamg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "paper_1102_0919_gb300: compiled library missing at %s; run "
        "`python -c 'import __graft_entry__ as g; g.build()'` first" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

OK, E_INVALID, E_NOMEM, E_CUDA, E_NT_TOO_SMALL, E_NOT_CONVERGED, E_TIMEOUT = range(7)
STATUS = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "CUDA", 4: "NT_TOO_SMALL", 5: "NOT_CONVERGED",
          6: "TIMEOUT"}
DOMINANT, MINIMAL = 0, 1
SVD, SPD_EIG = 0, 1
FP64, FP32, BF16 = 0, 1, 2


class SamgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_int32), ("theta", ctypes.c_double), ("mu_t", ctypes.c_int32),
                ("mu_b", ctypes.c_int32), ("mu_tJ", ctypes.c_int32), ("mu_bJ", ctypes.c_int32),
                ("omega_J", ctypes.c_double), ("n_mult", ctypes.c_int32),
                ("coarsest_max", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int), ("n_conv", ctypes.c_int32),
                ("coarse_pinv", ctypes.c_int32), ("row_form", ctypes.c_int32),
                ("relax_order", ctypes.c_int32), ("square_form", ctypes.c_int32),
                ("redo_tol", ctypes.c_double)]


class _Csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


_P = ctypes.c_void_p
_CTX = ctypes.c_void_p
_I = ctypes.c_int


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


samg_default_params = _sig("samg_default_params", None, ctypes.POINTER(Params))
samg_setup = _sig("samg_setup", _I, ctypes.POINTER(_Csr), _I, _I, _I, ctypes.POINTER(Params), _P,
                  ctypes.POINTER(_CTX))
samg_import = _sig("samg_import", _I, ctypes.POINTER(_Csr), _I, ctypes.POINTER(_Csr),
                   ctypes.POINTER(_Csr), _I, _I, _I, ctypes.POINTER(Params), _P, _P, _P, _P,
                   ctypes.POINTER(_CTX))
samg_destroy = _sig("samg_destroy", None, _CTX)
samg_last_error = _sig("samg_last_error", ctypes.c_char_p, _CTX)
samg_solve = _sig("samg_solve", _I, _CTX, ctypes.c_double, _I, ctypes.POINTER(_I))
samg_set_triplets = _sig("samg_set_triplets", _I, _CTX, _P, _P, _P)
samg_get_triplets = _sig("samg_get_triplets", _I, _CTX, _P, _P, _P, _P)
samg_set_precision = _sig("samg_set_precision", _I, _CTX, _I)
samg_set_coarse_pinv = _sig("samg_set_coarse_pinv", _I, _CTX, _I)
samg_set_relax_order = _sig("samg_set_relax_order", _I, _CTX, _I)
samg_get_hierarchy_info = _sig("samg_get_hierarchy_info", _I, _CTX, ctypes.POINTER(_I), _P, _P, _P)
samg_get_level_matrix = _sig("samg_get_level_matrix", _I, _CTX, _I, _I, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), _P, _P, _P)
samg_relax = _sig("samg_relax", _I, _CTX, _I, _I, _P, _P, _P, _P, _P)
samg_residual_restrict = _sig("samg_residual_restrict", _I, _CTX, _I, _P, _P, _P, _P, _P, _P, _P)
samg_interpolate = _sig("samg_interpolate", _I, _CTX, _I, _P, _P, _P, _P)
samg_coarsest_solve = _sig("samg_coarsest_solve", _I, _CTX, _P, _P, _P, _P, _P)
samg_vcycle = _sig("samg_vcycle", _I, _CTX, _P, _P, _P)
samg_ritz = _sig("samg_ritz", _I, _CTX, _P, _P, _P, _P)
samg_block_gram = _sig("samg_block_gram", _I, _P, _P, ctypes.c_int64, _I, _I, _P, _P)
samg_debug_mute_band = _sig("samg_debug_mute_band", _I, _CTX, _I, _I, _I)
samg_host_coarsen = _sig("samg_host_coarsen", _I, _P, ctypes.c_double, _P)
samg_host_ls_interp = _sig("samg_host_ls_interp", _I, _P, ctypes.c_double, _P, _I, _P, _P, _P,
                           ctypes.POINTER(ctypes.c_int64), _P, _P, _P)
_BATCH = ctypes.c_void_p
samg_setup_batched = _sig("samg_setup_batched", _I, _P, _I, _I, _I, _I, _P, ctypes.c_void_p,
                          ctypes.POINTER(_BATCH))
samg_solve_batched = _sig("samg_solve_batched", _I, _BATCH, ctypes.c_double, _I, _P)
samg_batch_problem = _sig("samg_batch_problem", _I, _BATCH, _I, ctypes.POINTER(_CTX))
samg_batch_size = _sig("samg_batch_size", _I, _BATCH)
samg_batch_last_error = _sig("samg_batch_last_error", ctypes.c_char_p, _BATCH)
samg_batch_destroy = _sig("samg_batch_destroy", None, _BATCH)
samg_export = _sig("samg_export", _I, _CTX, ctypes.c_char_p)
samg_write_hierarchy = _sig("samg_write_hierarchy", _I, ctypes.c_char_p, _P, _I, _P, _P, _I, _I, _I,
                            _P, _P, _P)
samg_import_file = _sig("samg_import_file", _I, ctypes.c_char_p, _P, ctypes.c_void_p,
                        ctypes.POINTER(_CTX))
samg_sweep_schedule = _sig("samg_sweep_schedule", _I, _P, _P, _P, _I, _I, _I, _I, _I, _P, ctypes.c_int64,
                           ctypes.POINTER(ctypes.c_int64))
samg_host_strength_product = _sig("samg_host_strength_product", _I, _P, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_int64), _P, _P, _P)
samg_sweep_plan = _sig("samg_sweep_plan", _I, _P, _I, _P, ctypes.c_int64, ctypes.POINTER(_I),
                       ctypes.POINTER(_I))
samg_block_gram_noalloc = _sig("samg_block_gram_noalloc", _I, _P, _P, ctypes.c_int64, _I, _I, _P,
                               _P)
samg_set_triplets_device = _sig("samg_set_triplets_device", _I, _CTX, _P, _P, _P)
samg_row_colours = _sig("samg_row_colours", _I, _P, _P, ctypes.POINTER(ctypes.c_int32))
samg_profile = _sig("samg_profile", _I, _CTX, _I)
samg_launch_count = _sig("samg_launch_count", ctypes.c_uint64)
samg_profile_read = _sig("samg_profile_read", _I, _CTX, _I, _I, ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))
samg_redo_interpolation = _sig("samg_redo_interpolation", _I, _CTX, _P)
samg_set_sweep_banding = _sig("samg_set_sweep_banding", _I, _CTX, _I, _I)
samg_set_sweep_banding_level = _sig("samg_set_sweep_banding_level", _I, _CTX, _I, _I)
samg_setup_times = _sig("samg_setup_times", _I, _CTX, _P, ctypes.c_int32)

EXPORTED = ["samg_default_params", "samg_setup", "samg_import", "samg_destroy", "samg_last_error",
            "samg_solve", "samg_set_triplets", "samg_get_triplets", "samg_set_precision",
            "samg_set_coarse_pinv", "samg_set_relax_order",
            "samg_get_hierarchy_info", "samg_get_level_matrix", "samg_relax",
            "samg_residual_restrict", "samg_interpolate", "samg_coarsest_solve", "samg_vcycle",
            "samg_ritz", "samg_block_gram", "samg_block_gram_noalloc", "samg_set_triplets_device",
            "samg_profile", "samg_profile_read", "samg_launch_count", "samg_debug_mute_band",
            "samg_sweep_plan", "samg_host_coarsen", "samg_host_ls_interp",
            "samg_host_strength_product", "samg_export", "samg_write_hierarchy",
            "samg_import_file", "samg_sweep_schedule", "samg_setup_batched",
            "samg_solve_batched", "samg_batch_problem", "samg_batch_size",
            "samg_batch_last_error", "samg_batch_destroy", "samg_row_colours",
            "samg_setup_times", "samg_redo_interpolation", "samg_set_sweep_banding",
            "samg_set_sweep_banding_level"]


def _arr(x, dtype):
    return None if x is None else np.ascontiguousarray(x, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(A):
    """Host CSR view of a scipy CSR matrix or workloads.CSR (arrays kept alive)."""
    if hasattr(A, "indptr"):
        A = A.tocsr()
        A.sort_indices()
        rp, ci, v, (m, n) = A.indptr, A.indices, A.data, A.shape
    else:
        rp, ci, v, m, n = A.row_ptr, A.col, A.val, A.m, A.n
    rp = _arr(rp, np.int64)
    ci = _arr(ci, np.int32)
    v = _arr(v, np.float64)
    c = _Csr(int(m), int(n), int(rp[-1]), _ptr(rp), _ptr(ci), _ptr(v))
    c._keep = (rp, ci, v)
    return c


def row_colours(A):
    """The library's greedy row colouring of A (host only): (colours, count)."""
    c = _csr(A)
    out = np.zeros(max(c.m, 1), np.int32)
    k = ctypes.c_int32(0)
    st = samg_row_colours(ctypes.byref(c), _ptr(out), ctypes.byref(k))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    return out[:c.m], k.value


def make_params(**kw) -> Params:
    p = Params()
    samg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "prec":
            v = {"fp64": FP64, "fp32": FP32, "bf16": BF16}.get(v, v)
        elif k == "coarse_pinv":
            v = {"svd": 0, "geneig": 1}.get(v, v)
        elif k == "row_form":
            v = {"induced": 0, "paper": 1}.get(v, v)
        elif k == "relax_order":
            v = {"natural": 0, "coloured": 1}.get(v, v)
        elif k == "square_form":
            v = {"normal": 0, "from_A": 1, "shared": 2}.get(v, v)
        setattr(p, k, v)
    return p


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


class Solver:
    """One solver context (owns its device memory)."""

    def __init__(self, ctx, nb, kind, target, m, n):
        self._ctx = ctx
        self.nb, self.kind, self.target, self.m, self.n = nb, kind, target, m, n

    # ---------------------------------------------------------- creation
    @classmethod
    def setup(cls, A, nb, target="minimal", kind="svd", stream=None, **params):
        t = MINIMAL if target == "minimal" else DOMINANT
        k = SPD_EIG if kind == "spd" else SVD
        c = _csr(A)
        p = make_params(**params)
        ctx = _CTX()
        st = samg_setup(ctypes.byref(c), nb, t, k, ctypes.byref(p), _stream(stream), ctypes.byref(ctx))
        if st != OK:
            raise SamgError(st, samg_last_error(None).decode())
        return cls(ctx, nb, k, t, c.m, c.n)

    @classmethod
    def from_hierarchy(cls, A, Ps, Qs, nb, sigma, U, V, target="minimal", kind="svd",
                       stream=None, **params):
        t = MINIMAL if target == "minimal" else DOMINANT
        k = SPD_EIG if kind == "spd" else SVD
        c = _csr(A)
        # the _Csr objects own the numpy arrays their pointers refer to; the
        # ctypes arrays below hold copies of the structs, so keep both alive
        Pl = [_csr(x) for x in Ps]
        P = (_Csr * len(Pl))(*Pl)
        if k == SVD:
            Ql = [_csr(x) for x in Qs]
            Q = (_Csr * len(Ql))(*Ql)
        else:
            Ql, Q = Pl, P
        p = make_params(**params)
        s = _arr(sigma, np.float64)
        u = _arr(U, np.float64)
        v = _arr(V, np.float64)
        ctx = _CTX()
        st = samg_import(ctypes.byref(c), len(Ps) + 1, P, Q, nb, t, k, ctypes.byref(p), _ptr(s),
                         _ptr(u), _ptr(v), _stream(stream), ctypes.byref(ctx))
        del Pl, Ql
        if st != OK:
            raise SamgError(st, samg_last_error(None).decode())
        return cls(ctx, nb, k, t, c.m, c.n)

    @classmethod
    def from_file(cls, path, stream=None, **params):
        """Context from a hierarchy file (samg_import_file)."""
        p = make_params(**params)
        ctx = _CTX()
        st = samg_import_file(os.fsencode(path), ctypes.byref(p), _stream(stream), ctypes.byref(ctx))
        if st != OK:
            raise SamgError(st, samg_last_error(None).decode())
        # n_b, kind, target and the finest shape from the file's header (the
        # library has just validated the whole file)
        with open(path, "rb") as f:
            head = f.read(36)
        kind, target, nb = np.frombuffer(head[12:24], dtype="<u4")
        m, n = np.frombuffer(head[28:36], dtype="<i4")
        return cls(ctx, int(nb), int(kind), int(target), int(m), int(n))

    def export(self, path):
        """Write the hierarchy and the current boot triplets (samg_export)."""
        self._check(samg_export(self._ctx, os.fsencode(path)))

    def close(self):
        if self._ctx and not getattr(self, "_borrowed", False):
            samg_destroy(self._ctx)
        self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise SamgError(st, samg_last_error(self._ctx).decode())

    # ---------------------------------------------------------- queries
    @property
    def spd(self):
        return self.kind == SPD_EIG

    @property
    def mu(self):
        return self.n if self.spd else self.m

    def levels(self):
        nl = ctypes.c_int(0)
        self._check(samg_get_hierarchy_info(self._ctx, ctypes.byref(nl), None, None, None))
        m = np.zeros(nl.value, np.int32)
        n = np.zeros(nl.value, np.int32)
        z = np.zeros(nl.value, np.int64)
        self._check(samg_get_hierarchy_info(self._ctx, ctypes.byref(nl), _ptr(m), _ptr(n), _ptr(z)))
        return [(int(a), int(b), int(c)) for a, b, c in zip(m, n, z)]

    def level_matrix(self, level, which):
        """(row_ptr, col, val, shape) of A_l (0), B_l (1), C_l (2), P_l (3), Q_l (4)."""
        w = {"A": 0, "B": 1, "C": 2, "P": 3, "Q": 4}.get(which, which)
        r, c, z = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        self._check(samg_get_level_matrix(self._ctx, level, w, ctypes.byref(r), ctypes.byref(c),
                                          ctypes.byref(z), None, None, None))
        rp = np.zeros(r.value + 1, np.int64)
        ci = np.zeros(max(z.value, 1), np.int32)
        v = np.zeros(max(z.value, 1), np.float64)
        self._check(samg_get_level_matrix(self._ctx, level, w, ctypes.byref(r), ctypes.byref(c),
                                          ctypes.byref(z), _ptr(rp), _ptr(ci), _ptr(v)))
        return rp, ci[:z.value], v[:z.value], (r.value, c.value)

    def set_precision(self, prec):
        self._check(samg_set_precision(self._ctx, {"fp64": FP64, "fp32": FP32, "bf16": BF16}.get(prec, prec)))

    def set_coarse_pinv(self, form):
        """0: the paper's SVD pseudo-inverse on the coarsest level; 1: the
        generalized-eigen variant."""
        self._check(samg_set_coarse_pinv(self._ctx, int(form)))

    def residuals(self):
        """rho_j of the current triplets (n_b values; no vector copies)."""
        r = np.zeros(self.nb)
        self._check(samg_get_triplets(self._ctx, None, None, None, _ptr(r)))
        return r

    def set_sweep_banding(self, band_rows=0, float_windows=False, level=None):
        """Rows per dependency level a sweep band grows to (0: the default
        per level), and whether float32 launches use programs with
        float32-only windows; with level, that level only."""
        if level is not None:
            self._check(samg_set_sweep_banding_level(self._ctx, int(level), int(band_rows)))
        else:
            self._check(samg_set_sweep_banding(self._ctx, int(band_rows), int(bool(float_windows))))

    def set_relax_order(self, order):
        """"natural" (0, the paper's) or "coloured" (1, the variant)."""
        self._check(samg_set_relax_order(self._ctx, {"natural": 0, "coloured": 1}.get(order, order)))

    # ---------------------------------------------------------- solve
    def solve(self, tol=1e-8, max_outer=100):
        done = ctypes.c_int(0)
        st = samg_solve(self._ctx, tol, max_outer, ctypes.byref(done))
        if st not in (OK, E_NOT_CONVERGED):
            self._check(st)
        return st == OK, done.value

    def triplets(self):
        s = np.zeros(self.nb)
        r = np.zeros(self.nb)
        U = np.zeros((self.mu, self.nb))
        V = None if self.spd else np.zeros((self.n, self.nb))
        self._check(samg_get_triplets(self._ctx, _ptr(s), _ptr(U), _ptr(V), _ptr(r)))
        return s, U, V, r

    def set_triplets(self, sigma, U, V=None):
        s, u, v = _arr(sigma, np.float64), _arr(U, np.float64), _arr(V, np.float64)
        self._check(samg_set_triplets(self._ctx, _ptr(s), _ptr(u), _ptr(v)))

    def set_triplets_device(self, sigma_ptr, U_ptr, V_ptr=None):
        """Device pointers (ints), row-major n_b columns."""
        self._check(samg_set_triplets_device(self._ctx, ctypes.c_void_p(sigma_ptr),
                                             ctypes.c_void_p(U_ptr),
                                             None if V_ptr is None else ctypes.c_void_p(V_ptr)))

    KERNELS = ("kaczmarz_sweep", "block_spmm", "jacobi", "coarsest_solve", "ritz")

    SETUP_STAGES = ("strength_rs", "test_relax", "boot_relax", "ls_fit", "galerkin",
                    "prepare_level", "coarsest", "ritz", "finalize", "other")

    def redo_interpolation(self, converged):
        """Sec. 6.3: new P and Q by one downward sweep, the LS weights of the
        test vectors and of the converged triplets divided by 1000."""
        c = np.ascontiguousarray(np.asarray(converged, dtype=np.int32))
        assert c.size == self.nb
        self._check(samg_redo_interpolation(self._ctx, _ptr(c)))

    def setup_times(self):
        """Wall seconds of the last setup's stages (strength and splitting,
        test and boot relaxation, LS fits, Galerkin, level preparation,
        coarsest solve, Ritz, completion, the rest)."""
        t = np.zeros(len(self.SETUP_STAGES))
        self._check(samg_setup_times(self._ctx, _ptr(t), len(t)))
        return dict(zip(self.SETUP_STAGES, (float(x) for x in t)))

    def profile(self, on=True):
        self._check(samg_profile(self._ctx, 1 if on else 0))

    def profile_read(self, reset=True):
        out = {}
        for k, name in enumerate(self.KERNELS):
            n, ms, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            self._check(samg_profile_read(self._ctx, k, 1 if (reset and k == 4) else 0,
                                          ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)))
            out[name] = dict(launches=n.value, ms=ms.value, bytes=b.value)
        return out

    def debug_mute_band(self, level, which, band):
        """Test hook: band `band` of level `level`'s sweep over the rows of A
        (which 0), of A^t (1), or of every fused relaxation program built so
        far (2) stops publishing its progress (-1 restores)."""
        self._check(samg_debug_mute_band(self._ctx, level, which, band))

    # ---------------------------------------------------------- single steps
    def relax(self, level, sigma, U, V, K=None, T=None, count=1):
        U = np.array(U, dtype=np.float64, order="C")
        V = None if V is None else np.array(V, dtype=np.float64, order="C")
        s, k, t = _arr(sigma, np.float64), _arr(K, np.float64), _arr(T, np.float64)
        self._check(samg_relax(self._ctx, level, count, _ptr(s), _ptr(U), _ptr(V), _ptr(k), _ptr(t)))
        return U, V

    def residual_restrict(self, level, sigma, U, V, K, T, mc, nc):
        s, u, v, k, t = (_arr(x, np.float64) for x in (sigma, U, V, K, T))
        Kc = np.zeros((mc, self.nb))
        Tc = None if self.spd else np.zeros((nc, self.nb))
        self._check(samg_residual_restrict(self._ctx, level, _ptr(s), _ptr(u), _ptr(v), _ptr(k),
                                           _ptr(t), _ptr(Kc), _ptr(Tc)))
        return Kc, Tc

    def interpolate(self, level, U, V, Uc, Vc):
        U = np.array(U, dtype=np.float64, order="C")
        V = None if V is None else np.array(V, dtype=np.float64, order="C")
        uc, vc = _arr(Uc, np.float64), _arr(Vc, np.float64)
        self._check(samg_interpolate(self._ctx, level, _ptr(U), _ptr(V), _ptr(uc), _ptr(vc)))
        return U, V

    def coarsest_solve(self, sigma, K, T, mL, nL):
        s, k, t = _arr(sigma, np.float64), _arr(K, np.float64), _arr(T, np.float64)
        U = np.zeros((mL, self.nb))
        V = None if self.spd else np.zeros((nL, self.nb))
        self._check(samg_coarsest_solve(self._ctx, _ptr(s), _ptr(k), _ptr(t), _ptr(U), _ptr(V)))
        return U, V

    def vcycle(self, sigma, U, V=None):
        U = np.array(U, dtype=np.float64, order="C")
        V = None if V is None else np.array(V, dtype=np.float64, order="C")
        s = _arr(sigma, np.float64)
        self._check(samg_vcycle(self._ctx, _ptr(s), _ptr(U), _ptr(V)))
        return U, V

    def ritz(self, U, V=None):
        U = np.array(U, dtype=np.float64, order="C")
        V = None if V is None else np.array(V, dtype=np.float64, order="C")
        s = np.zeros(self.nb)
        r = np.zeros(self.nb)
        self._check(samg_ritz(self._ctx, _ptr(s), _ptr(U), _ptr(V), _ptr(r)))
        return s, U, V, r


def block_gram(X_ptr, Y_ptr, rows, nb, ld, G_ptr, stream=None):
    """G = X^t Y for device blocks (raw device pointers as ints)."""
    st = samg_block_gram(ctypes.c_void_p(X_ptr), ctypes.c_void_p(Y_ptr), rows, nb, ld,
                         ctypes.c_void_p(G_ptr), _stream(stream))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())


def block_gram_noalloc(X_ptr, Y_ptr, rows, nb, ld, G_ptr, stream=None):
    """G = X^t Y like block_gram, with the partial sums in the library's fixed
    device scratch (no allocation, no stream synchronization).  Calls whose GPU
    work overlaps race on that scratch; rows are limited to
    ceil(rows / 4096) * nb * nb <= 65536."""
    st = samg_block_gram_noalloc(ctypes.c_void_p(X_ptr), ctypes.c_void_p(Y_ptr), rows, nb, ld,
                                 ctypes.c_void_p(G_ptr), _stream(stream))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())


def sweep_plan(A, fused_count=0):
    """Host-only: (row levels, depth, bands) of the exact-order Kaczmarz
    schedule of one sweep over the rows of A (fused_count 0) or of
    fused_count fused minimal-SVD relaxations with B = C = I."""
    c = _csr(A)
    rows = c.m if fused_count == 0 else fused_count * (c.m + c.n)
    lv = np.zeros(max(rows, 1), np.int32)
    d, nb = ctypes.c_int(0), ctypes.c_int(0)
    st = samg_sweep_plan(ctypes.byref(c), fused_count, _ptr(lv), lv.size, ctypes.byref(d),
                         ctypes.byref(nb))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    return lv[:rows], d.value, nb.value


def sweep_schedule(A, fused_count=0, spd=False, B=None, C=None, resident_slots=0, band_rows=0,
                   slot_cap=0):
    """Host-only: the serialized sweep schedule (bytes) the kernels receive
    (B, C: the level's operators; None = identity; resident_slots > 0: one
    resident band when the program keeps at most that many columns live;
    band_rows: rows per level a band grows to, 0 = 32; slot_cap: live
    columns per band, 0 = 512)."""
    c = _csr(A)
    cb = None if B is None else _csr(B)
    cc = None if C is None else _csr(C)
    args = (ctypes.byref(c), None if cb is None else ctypes.byref(cb),
            None if cc is None else ctypes.byref(cc), fused_count, int(spd), int(resident_slots),
            int(band_rows), int(slot_cap))
    size = ctypes.c_int64(0)
    st = samg_sweep_schedule(*args, None, 0, ctypes.byref(size))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    buf = np.zeros(size.value, np.uint8)
    st = samg_sweep_schedule(*args, _ptr(buf), size.value, ctypes.byref(size))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    return buf.tobytes()


def host_coarsen(N, theta):
    """Host-only: C/F splitting (1 = C) of the strength graph of N."""
    c = _csr(N)
    cf = np.zeros(c.m, np.int8)
    st = samg_host_coarsen(ctypes.byref(c), theta, _ptr(cf))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    return cf


class Batch:
    """Independent problems with one n_b, target, kind and parameter set
    (samg_setup_batched); problem(i) is a Solver view owned by the batch."""

    def __init__(self, b, nb, kind, target, shapes):
        self._b = b
        self.nb, self.kind, self.target, self.shapes = nb, kind, target, shapes

    @classmethod
    def setup(cls, As, nb, target="minimal", kind="svd", stream=None, **params):
        t = MINIMAL if target == "minimal" else DOMINANT
        k = SPD_EIG if kind == "spd" else SVD
        cs = [_csr(A) for A in As]
        ptrs = (ctypes.c_void_p * len(cs))(*[ctypes.cast(ctypes.pointer(c), ctypes.c_void_p)
                                             for c in cs])
        p = make_params(**params)
        b = _BATCH()
        st = samg_setup_batched(ptrs, len(cs), nb, t, k, ctypes.byref(p), _stream(stream),
                                ctypes.byref(b))
        if st != OK:
            raise SamgError(st, samg_batch_last_error(None).decode())
        return cls(b, nb, k, t, [(c.m, c.n) for c in cs])

    def solve(self, tol=1e-8, max_outer=100):
        done = np.zeros(len(self.shapes), np.int32)
        st = samg_solve_batched(self._b, tol, max_outer, _ptr(done))
        if st not in (OK, E_NOT_CONVERGED):
            raise SamgError(st, samg_batch_last_error(self._b).decode())
        return st == OK, done

    def problem(self, i):
        ctx = _CTX()
        if samg_batch_problem(self._b, i, ctypes.byref(ctx)) != OK:
            raise SamgError(E_INVALID, "no problem %d" % i)
        m, n = self.shapes[i]
        v = Solver(ctx, self.nb, self.kind, self.target, m, n)
        v._borrowed = True
        return v

    def close(self):
        if self._b:
            samg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def write_hierarchy(path, A, Ps, Qs, sigma, U, V, target="minimal", kind="svd"):
    """Host-only: write a hierarchy file from host arrays (samg_write_hierarchy)."""
    t = MINIMAL if target == "minimal" else DOMINANT
    k = SPD_EIG if kind == "spd" else SVD
    c = _csr(A)
    Pl = [_csr(x) for x in Ps]
    P = (_Csr * len(Pl))(*Pl)
    Ql = [_csr(x) for x in Qs] if k == SVD else []
    Q = (_Csr * len(Ql))(*Ql) if Ql else None
    s = _arr(sigma, np.float64)
    u = _arr(U, np.float64)
    v = _arr(V, np.float64) if k == SVD else None
    st = samg_write_hierarchy(os.fsencode(path), ctypes.byref(c), len(Ps) + 1, P, Q, len(s), t, k,
                              _ptr(s), _ptr(u), _ptr(v))
    del Pl, Ql
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())


def host_strength_product(A, theta):
    """Host-only: strong influences of A A^t (scipy CSR, values |n_ij|),
    computed from A without forming the product."""
    import scipy.sparse as _sp

    c = _csr(A)
    nnz = ctypes.c_int64(0)
    st = samg_host_strength_product(ctypes.byref(c), theta, ctypes.byref(nnz), None, None, None)
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    rp = np.zeros(c.m + 1, np.int64)
    ci = np.zeros(max(nnz.value, 1), np.int32)
    v = np.zeros(max(nnz.value, 1), np.float64)
    st = samg_host_strength_product(ctypes.byref(c), theta, ctypes.byref(nnz), _ptr(rp), _ptr(ci),
                                    _ptr(v))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    return _sp.csr_matrix((v[:nnz.value], ci[:nnz.value], rp), shape=(c.m, c.m))


def host_ls_interp(N, theta, cf, Yf, Yc, w):
    """Host-only: the setup's LS interpolation operator (scipy CSR)."""
    import scipy.sparse as _sp

    c = _csr(N)
    nf = int(np.asarray(Yf).shape[1])
    cf8 = np.ascontiguousarray(cf, dtype=np.int8)
    f = _arr(Yf, np.float64)
    g = _arr(Yc, np.float64)
    ww = _arr(w, np.float64)
    nnz = ctypes.c_int64(0)
    args = (ctypes.byref(c), theta, _ptr(cf8), nf, _ptr(f), _ptr(g), _ptr(ww), ctypes.byref(nnz))
    st = samg_host_ls_interp(*args, None, None, None)
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    rp = np.zeros(c.m + 1, np.int64)
    ci = np.zeros(max(nnz.value, 1), np.int32)
    v = np.zeros(max(nnz.value, 1), np.float64)
    st = samg_host_ls_interp(*args, _ptr(rp), _ptr(ci), _ptr(v))
    if st != OK:
        raise SamgError(st, samg_last_error(None).decode())
    return _sp.csr_matrix((v[:nnz.value], ci[:nnz.value], rp), shape=(c.m, int(cf8.sum())))
