"""ctypes binding of libdmrg.so: same names as the C-ABI, argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

DMRG_FP64, DMRG_BF16X3, DMRG_BF16, DMRG_BF16X6, DMRG_FP64_TC = 0, 1, 2, 3, 4
DMRG_PRECOND_JACOBI, DMRG_PRECOND_MLP = 0, 1
STATUS = {0: "DMRG_OK", -1: "DMRG_EINVAL", -2: "DMRG_ENOMEM", -3: "DMRG_ECUDA", -4: "DMRG_ENUMERIC",
          -5: "DMRG_ETIMEOUT", -6: "DMRG_ENOTCONV", -7: "DMRG_EIO"}


class DMRGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("n_roots", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("max_space", C.c_int), ("precond", C.c_int), ("fp64_final", C.c_int),
                ("mem_budget", C.c_int64), ("scratch_bytes", C.c_int64), ("keep_envs", C.c_int),
                ("verbose", C.c_int), ("tc_kchunk", C.c_int64), ("fp64_store", C.c_int), ("sigma_graph", C.c_int),
                ("sigma_tune", C.c_int), ("sigma_tile_n", C.c_int), ("refine", C.c_int), ("max_refine", C.c_int),
                ("fp64_tc", C.c_int), ("host_tier", C.c_int),
                ("sigma_per_term", C.c_int), ("decim_tol32", C.c_double),
                ("decim_fp64_units", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("sigma_calls", C.c_int64), ("sigma_flops", C.c_double), ("sigma_ms_last", C.c_double),
                ("interm_flops", C.c_double), ("renorm_flops_last", C.c_double),
                ("ms_interm", C.c_double), ("ms_gemm", C.c_double), ("ms_renorm", C.c_double),
                ("ms_davidson", C.c_double), ("ms_decim", C.c_double), ("ms_hdiag", C.c_double),
                ("n_terms", C.c_int64), ("n_items", C.c_int64), ("store_bytes", C.c_int64),
                ("interm_bytes", C.c_int64), ("device_bytes", C.c_int64), ("kernel_launches", C.c_int64),
                ("precond_fallbacks", C.c_int64), ("davidson_iters_last", C.c_int),
                ("ms_host_plan", C.c_double), ("sigma_tiles", C.c_int64 * 2), ("sigma_stages", C.c_int64 * 2),
                ("sigma_mma_flops", C.c_double), ("sigma_maps", C.c_int64), ("ms_decim_parts", C.c_double * 4),
                ("decim_sweeps_last", C.c_int), ("ms_sigma_dev", C.c_double), ("sigma_flops_dev", C.c_double),
                ("sigma_stages_dev", C.c_int64), ("sigma_timed", C.c_int64), ("decim_conv_last", C.c_double * 41),
                ("decim_nmat_last", C.c_int), ("decim_nmax_last", C.c_int), ("decim_sweeps32_last", C.c_int),
                ("sigma_tile_n", C.c_int),
                ("sigma_kchunk", C.c_int64), ("tunes", C.c_int64), ("tune_hits", C.c_int64), ("ms_tune", C.c_double),
                ("tune_cand_ms", C.c_double * 4), ("sigma_load_bytes", (C.c_double * 2) * 2),
                ("renorm_flops_total", C.c_double), ("interm_flops_total", C.c_double),
                ("davidson_rnorm_last", C.c_double), ("davidson_conv_last", C.c_int),
                ("davidson_stalled_last", C.c_int), ("davidson_refine_last", C.c_int), ("sigma_chunks", C.c_int),
                ("sigma_acc_calls", C.c_int64), ("ms_sigma_acc", C.c_double), ("sigma_acc_flops", C.c_double),
                ("device_bytes_peak", C.c_int64), ("host_bytes", C.c_int64), ("tier_out_bytes", C.c_int64),
                ("tier_in_bytes", C.c_int64), ("ms_tier_wait", C.c_double)]

    def as_dict(self):
        def conv(v):
            return [conv(x) for x in v] if isinstance(v, C.Array) else v

        return {f: conv(getattr(self, f)) for f, _ in self._fields_}


def lib_path():
    return os.path.join(HERE, "libdmrg.so")


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_int64)

_SIGS = {
    "dmrg_default_options": (None, [C.POINTER(Options)]),
    "dmrg_version": (C.c_char_p, []),
    "dmrg_plan": (C.c_int, [_D, _D, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                            C.POINTER(Options), C.c_char_p, C.POINTER(_P)]),
    "dmrg_set_bond": (C.c_int, [_P, C.c_int, _P]),
    "dmrg_layout": (C.c_int, [_P, _L, _I, _L, _I]),
    "dmrg_sigma": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dmrg_sigma_host": (C.c_int, [_P, _D, _D, C.c_int, _P]),
    "dmrg_sigma_fp64": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dmrg_sigma_fp64_units": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dmrg_hdiag": (C.c_int, [_P, _P, _P]),
    "dmrg_davidson": (C.c_int, [_P, _P, C.c_int, C.c_double, C.c_int, C.c_int, _D, _I, _P]),
    "dmrg_decimate": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, _D, _P, _L, _P]),
    "dmrg_update_bond_host": (C.c_int, [_P, _D, C.c_int, C.c_int, C.c_int, _D, _I, _D, _D, _L, _P]),
    "dmrg_set_refine": (C.c_int, [_P, C.c_int, C.c_int]),
    "dmrg_sweep": (C.c_int, [_P, C.c_int, _I, _D, _D, _P]),
    "dmrg_save_mps": (C.c_int, [_P, C.c_char_p]),
    "dmrg_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "dmrg_last_error": (C.c_char_p, [_P]),
    "dmrg_destroy": (None, [_P]),
    "dmrg_grouped_gemm": (C.c_int, [C.c_int, C.c_int, _I, _I, _L, _I, _I, _L, _I, _I, _L, _I, _I, _D,
                                    _P, _P, _P, _P]),
    "dmrg_grouped_gemm_noalloc": (C.c_int, [C.c_int, _I, _I, _L, _I, _I, _L, _I, _I, _L, _I, _I, _D,
                                            _P, _P, _P, _P]),
    "dmrg_noalloc_scratch_bytes": (C.c_int64, []),
    "dmrg_mlp_init": (C.c_int, [_P, C.c_uint32]),
    "dmrg_mlp_harvest": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int64, _D, _L, _P]),
    "dmrg_mlp_train": (C.c_int, [_P, C.c_int, C.c_int64, C.c_float, C.c_uint64, C.POINTER(C.c_float),
                                 C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float), _P]),
    "dmrg_mlp_eval": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, _P]),
    "dmrg_mlp_gradient": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P, _P, _P]),
    "dmrg_mlp_params": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int]),
    "dmrg_mlp_num_params": (C.c_int, []),
    "dmrg_extrapolate": (C.c_int, [_D, _D, C.c_int, _D, _D, _D]),
    "dmrg_selftest_wait": (C.c_int, [C.c_double, C.c_int, _P]),
}


def lib():
    """Load libdmrg.so from the package directory (raises if it is missing)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libdmrg.so not built ({path}); run python -m paper_2311_02854_gb300.build")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def version():
    return lib().dmrg_version().decode()


def _ptr(x):
    """Raw pointer of a torch tensor, numpy array or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _dptr(a):
    return a.ctypes.data_as(_D)


def _check(code, plan_handle=None):
    if code != 0:
        msg = lib().dmrg_last_error(plan_handle).decode()
        raise DMRGError(code, msg)


def default_options(**kw):
    o = Options()
    lib().dmrg_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


class Plan:
    """dmrg_plan: integrals + MPS file -> plan.  ``chol`` is either the
    Cholesky vectors (n_chol x K x K) or the full (pq|rs) array (K x K x K x K).
    ``close()`` calls dmrg_destroy."""

    def __init__(self, h, chol, K, N, twoS, D, mps_path, e_core=0.0, options=None, **kw):
        L = lib()
        self._h = np.ascontiguousarray(h, dtype=np.float64)
        self._chol = np.ascontiguousarray(chol, dtype=np.float64)
        opts = options if options is not None else default_options(**kw)
        self.options = opts
        handle = _P()
        # a 4-index array is the full (pq|rs) (n_chol = 0), else Cholesky vectors
        n_chol = 0 if self._chol.ndim == 4 else int(self._chol.shape[0])
        code = L.dmrg_plan(_dptr(self._h), _dptr(self._chol), n_chol, float(e_core),
                           int(K), int(N), int(twoS), int(D), C.byref(opts), str(mps_path).encode(),
                           C.byref(handle))
        _check(code, None)
        self.handle = handle
        self.K, self.N, self.twoS = K, N, twoS

    def close(self):
        if getattr(self, "handle", None):
            lib().dmrg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        code = getattr(lib(), name)(self.handle, *args)
        _check(code, self.handle)
        return code

    def set_bond(self, k, stream=None):
        self._call("dmrg_set_bond", int(k), _stream(stream))

    def layout(self):
        dim = C.c_int64()
        ns = C.c_int()
        self._call("dmrg_layout", C.byref(dim), C.byref(ns), None, None)
        offs = np.zeros(ns.value + 1, dtype=np.int64)
        qn = np.zeros(6 * ns.value, dtype=np.int32)
        self._call("dmrg_layout", C.byref(dim), C.byref(ns), offs.ctypes.data_as(_L),
                   qn.ctypes.data_as(_I))
        return dim.value, offs, qn.reshape(-1, 6)

    @property
    def dim(self):
        return self.layout()[0]

    def sigma(self, psi, out, nvec=1, stream=None):
        self._call("dmrg_sigma", _ptr(psi), _ptr(out), int(nvec), _stream(stream))

    def sigma_fp64(self, psi, out, nvec=1, stream=None):
        self._call("dmrg_sigma_fp64", _ptr(psi), _ptr(out), int(nvec), _stream(stream))

    def sigma_fp64_units(self, psi, out, nvec=1, stream=None):
        self._call("dmrg_sigma_fp64_units", _ptr(psi), _ptr(out), int(nvec), _stream(stream))

    def sigma_host(self, psi, out, nvec=1, stream=None):
        assert psi.dtype == np.float64 and out.dtype == np.float64
        self._call("dmrg_sigma_host", _dptr(psi), _dptr(out), int(nvec), _stream(stream))

    def hdiag(self, out, stream=None):
        self._call("dmrg_hdiag", _ptr(out), _stream(stream))

    def davidson(self, psi, n_roots=1, tol=1e-6, max_iter=200, precond=DMRG_PRECOND_JACOBI, stream=None):
        e = np.zeros(n_roots)
        it = C.c_int()
        code = getattr(lib(), "dmrg_davidson")(self.handle, _ptr(psi), int(n_roots), float(tol), int(max_iter),
                                                int(precond), _dptr(e), C.byref(it), _stream(stream))
        if code not in (0, -6):
            _check(code, self.handle)
        return e, it.value, code == 0

    def decimate(self, psi, n_roots, D, forward, next_psi=None, next_cap=0, stream=None):
        w = np.zeros(1)
        nd = C.c_int64(int(next_cap))
        self._call("dmrg_decimate", _ptr(psi), int(n_roots), int(D), int(bool(forward)), _dptr(w),
                   _ptr(next_psi), C.byref(nd), _stream(stream))
        return float(w[0]), nd.value

    def set_refine(self, refine, max_refine=0):
        self._call("dmrg_set_refine", int(bool(refine)), int(max_refine))

    def update_bond_host(self, psi, n_roots, D, forward, next_psi=None, stream=None):
        """dmrg_update_bond_host: Davidson + decimation from host buffers (numpy
        FP64 arrays; pinned memory if they view a pinned torch tensor).  Returns
        (energies, iterations, discarded weight, next dim, converged)."""
        assert psi.dtype == np.float64 and psi.flags.c_contiguous
        e = np.zeros(n_roots)
        it = C.c_int()
        w = np.zeros(1)
        cap = 0 if next_psi is None else int(next_psi.size // max(n_roots, 1))
        nd = C.c_int64(cap)
        nptr = None if next_psi is None else next_psi.ctypes.data_as(_D)
        code = getattr(lib(), "dmrg_update_bond_host")(self.handle, _dptr(psi), int(n_roots), int(D),
                                                        int(bool(forward)), _dptr(e), C.byref(it), _dptr(w), nptr,
                                                        C.byref(nd), _stream(stream))
        if code not in (0, -6):
            _check(code, self.handle)
        return e, it.value, float(w[0]), nd.value, code == 0

    def sweep(self, n_sweeps, D_schedule=None, stream=None):
        e = np.zeros(n_sweeps)
        w = np.zeros(n_sweeps)
        ds = None
        if D_schedule is not None:
            arr = np.ascontiguousarray(D_schedule, dtype=np.int32)
            ds = arr.ctypes.data_as(_I)
        code = getattr(lib(), "dmrg_sweep")(self.handle, int(n_sweeps), ds, _dptr(e), _dptr(w), _stream(stream))
        if code not in (0, -6):
            _check(code, self.handle)
        return e, w

    def save_mps(self, path):
        self._call("dmrg_save_mps", str(path).encode())

    def stats(self):
        s = Stats()
        self._call("dmrg_stats", C.byref(s))
        return s.as_dict()

    # --- learned Davidson preconditioner -----------------------------------
    def mlp_init(self, seed=3):
        self._call("dmrg_mlp_init", int(seed))

    def mlp_harvest(self, psi, max_iter=40, jd_iters=40, per_solve=1 << 14, stream=None):
        """Plain Davidson at the current bond collecting Jacobi-Davidson pairs;
        returns (energy, pairs added)."""
        e = C.c_double(0.0)
        n = C.c_int64(0)
        self._call("dmrg_mlp_harvest", _ptr(psi), int(max_iter), int(jd_iters), int(per_solve), C.byref(e),
                   C.byref(n), _stream(stream))
        return e.value, n.value

    def mlp_train(self, steps=400, batch=4096, lr=3e-3, seed=3, stream=None, held_out=False):
        """Adam on the collected pairs (weighted loss); returns the (first, last)
        training-batch loss, and with held_out=True also the (before, after)
        loss of the held-out last tenth of the pairs."""
        l0, l1, h0, h1 = C.c_float(0.0), C.c_float(0.0), C.c_float(0.0), C.c_float(0.0)
        self._call("dmrg_mlp_train", int(steps), int(batch), float(lr), int(seed), C.byref(l0), C.byref(l1),
                   C.byref(h0), C.byref(h1), _stream(stream))
        if held_out:
            return l0.value, l1.value, h0.value, h1.value
        return l0.value, l1.value

    def mlp_eval(self, x, g, bf16=False, stream=None):
        """g[i] = MLP(x[i, :5]) for device FP32 tensors."""
        n = int(x.numel() // 5)
        self._call("dmrg_mlp_eval", _ptr(x), n, _ptr(g), int(bool(bf16)), _stream(stream))

    def mlp_gradient(self, x, y, grad, loss, w=None, stream=None):
        n = int(x.numel() // 5)
        self._call("dmrg_mlp_gradient", _ptr(x), _ptr(y), _ptr(w), n, _ptr(grad), _ptr(loss), _stream(stream))

    def mlp_params(self, values=None):
        """Get (values None) or set the FP32 parameters (numpy float32 array)."""
        n = int(lib().dmrg_mlp_num_params())
        if values is None:
            out = np.zeros(n, dtype=np.float32)
            self._call("dmrg_mlp_params", out.ctypes.data_as(C.POINTER(C.c_float)), 0)
            return out
        arr = np.ascontiguousarray(values, dtype=np.float32)
        assert arr.size == n
        self._call("dmrg_mlp_params", arr.ctypes.data_as(C.POINTER(C.c_float)), 1)


def grouped_gemm(precision, blocks, a, b, c, stream=None):
    """dmrg_grouped_gemm.  ``blocks``: list of (m, n, c_off, [segments]) with
    segment = (k, a_off, lda, a_tr, b_off, ldb, b_tr, alpha); a, b, c device FP64."""
    ms, ns, coff, beg = [], [], [], [0]
    k, ao, la, at, bo, lb, bt, al = [], [], [], [], [], [], [], []
    for (m, n, co, segs) in blocks:
        ms.append(m)
        ns.append(n)
        coff.append(co)
        for s in segs:
            k.append(s[0]); ao.append(s[1]); la.append(s[2]); at.append(s[3])
            bo.append(s[4]); lb.append(s[5]); bt.append(s[6]); al.append(s[7])
        beg.append(len(k))
    i32 = lambda v: np.ascontiguousarray(v, dtype=np.int32)  # noqa: E731
    i64 = lambda v: np.ascontiguousarray(v, dtype=np.int64)  # noqa: E731
    arrs = [i32(ms), i32(ns), i64(coff), i32(beg), i32(k), i64(ao), i32(la), i32(at), i64(bo), i32(lb), i32(bt)]
    alpha = np.ascontiguousarray(al, dtype=np.float64)
    ptrs = [x.ctypes.data_as(_L if x.dtype == np.int64 else _I) for x in arrs]
    code = lib().dmrg_grouped_gemm(int(precision), len(ms), *ptrs, alpha.ctypes.data_as(_D), _ptr(a), _ptr(b),
                                   _ptr(c), _stream(stream))
    _check(code, None)


def grouped_gemm_noalloc(blocks, a, b, c, stream=None):
    """dmrg_grouped_gemm_noalloc: the FP64 grouped GEMM with its work list in a
    static device array, so the call allocates no device memory.  ``blocks`` as
    for grouped_gemm."""
    ms, ns, coff, beg = [], [], [], [0]
    k, ao, la, at, bo, lb, bt, al = [], [], [], [], [], [], [], []
    for (m, n, co, segs) in blocks:
        ms.append(m)
        ns.append(n)
        coff.append(co)
        for s in segs:
            k.append(s[0]); ao.append(s[1]); la.append(s[2]); at.append(s[3])
            bo.append(s[4]); lb.append(s[5]); bt.append(s[6]); al.append(s[7])
        beg.append(len(k))
    arrs = [np.ascontiguousarray(ms, dtype=np.int32), np.ascontiguousarray(ns, dtype=np.int32),
            np.ascontiguousarray(coff, dtype=np.int64), np.ascontiguousarray(beg, dtype=np.int32),
            np.ascontiguousarray(k, dtype=np.int32), np.ascontiguousarray(ao, dtype=np.int64),
            np.ascontiguousarray(la, dtype=np.int32), np.ascontiguousarray(at, dtype=np.int32),
            np.ascontiguousarray(bo, dtype=np.int64), np.ascontiguousarray(lb, dtype=np.int32),
            np.ascontiguousarray(bt, dtype=np.int32)]
    alpha = np.ascontiguousarray(al, dtype=np.float64)
    ptrs = [x.ctypes.data_as(_L if x.dtype == np.int64 else _I) for x in arrs]
    code = lib().dmrg_grouped_gemm_noalloc(len(ms), *ptrs, alpha.ctypes.data_as(_D), _ptr(a), _ptr(b), _ptr(c),
                                           _stream(stream))
    _check(code, None)


def extrapolate(w, E):
    """dmrg_extrapolate: least-squares line E = A w + E0 through a series of
    (discarded weight, energy) points; returns (E0, A, rms residual).  Host
    arithmetic in the library (no GPU needed)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    if w.shape != E.shape or w.ndim != 1:
        raise ValueError("w and E must be 1-D and equally long")
    e0, a, r = C.c_double(), C.c_double(), C.c_double()
    code = lib().dmrg_extrapolate(_dptr(w), _dptr(E), int(w.size), C.pointer(e0), C.pointer(a), C.pointer(r))
    _check(code, None)
    return e0.value, a.value, r.value


def selftest_wait(seconds, arrive, stream=None):
    """dmrg_selftest_wait: one bounded device wait on an mbarrier that is
    arrived on (``arrive``) or not; raises DMRGError(DMRG_ETIMEOUT) when the
    wait gave up."""
    _check(lib().dmrg_selftest_wait(float(seconds), int(arrive), _stream(stream)), None)


def noalloc_scratch_bytes():
    """Size of the static work-list array of grouped_gemm_noalloc."""
    return int(lib().dmrg_noalloc_scratch_bytes())
