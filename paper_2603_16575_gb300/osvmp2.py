"""Python binding of libosvmp2 (C ABI in include/osvmp2.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory and streams; the
library never falls back to a CPU path -- if ``libosvmp2.so`` is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libosvmp2.so")

OSVMP2_FP64 = 0
OSVMP2_MIXED = 1
PREC = {"fp64": OSVMP2_FP64, "mixed": OSVMP2_MIXED}

STATUS = {0: "OK", 1: "E_ARG", 2: "E_CUDA", 3: "E_NOMEM", 4: "E_NOCONV", 5: "E_NUMERIC", 6: "E_STATE",
          7: "E_TIMEOUT"}
STATUS_CODES = {v: k for k, v in STATUS.items()}


class Opts(ctypes.Structure):
    _fields_ = [("tau_s", ctypes.c_double), ("tol_update", ctypes.c_double), ("tol_energy", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("osv_prec", ctypes.c_int32), ("no_autotune", ctypes.c_int32),
                ("mem_cap_mib", ctypes.c_int32), ("osv_method", ctypes.c_int32), ("rosv_max_rows", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class System(ctypes.Structure):
    _fields_ = [("n_occ", ctypes.c_int32), ("n_vir", ctypes.c_int32), ("n_aux", ctypes.c_int32),
                ("B", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("env", ctypes.c_void_p),
                ("f_occ", ctypes.c_void_p), ("e_vir", ctypes.c_void_p), ("r_occ", ctypes.c_void_p)]


class MbeStats(ctypes.Structure):
    _fields_ = [("n_single", ctypes.c_int64), ("n_pair", ctypes.c_int64), ("n_triple", ctypes.c_int64),
                ("n_pair_blocks", ctypes.c_int64), ("max_iter_used", ctypes.c_int32),
                ("n_unconverged", ctypes.c_int32), ("worst_fragment", ctypes.c_int64),
                ("max_update", ctypes.c_double), ("flops", ctypes.c_double), ("n_weak", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Screen(ctypes.Structure):
    """Pair-class cuts (paper defaults 1e-7, 1e-2, 0.2)."""
    _fields_ = [("s2b_distant", ctypes.c_double), ("s2b_close", ctypes.c_double), ("s3b_min", ctypes.c_double)]

    def __init__(self, s2b_distant=1e-7, s2b_close=1e-2, s3b_min=0.2):
        super().__init__(s2b_distant, s2b_close, s3b_min)


# name -> (restype, argtypes); every function declared in include/osvmp2.h
_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "osvmp2_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.POINTER(Opts)]),
    "osvmp2_destroy": (None, [_P]),
    "osvmp2_last_error": (ctypes.c_char_p, [_P]),
    "osvmp2_default_opts": (None, [ctypes.POINTER(Opts)]),
    "osvmp2_set_opts": (ctypes.c_int, [_P, ctypes.POINTER(Opts)]),
    "osvmp2_get_solve_plan": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "osvmp2_kernel_launches": (ctypes.c_int64, []),
    "osvmp2_build_osv": (ctypes.c_int, [_P, ctypes.POINTER(System), _D, _P]),
    "osvmp2_get_osv": (ctypes.c_int, [_P, _I32, _P, _P]),
    "osvmp2_pair_integrals": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int]),
    "osvmp2_get_pair_blocks": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P]),
    "osvmp2_get_precond": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P]),
    "osvmp2_solve": (ctypes.c_int, [_P, _P, _I32, ctypes.c_int, _P, _P, _P]),
    "osvmp2_mbe3_energy": (ctypes.c_int, [_P, _D, _D, ctypes.c_int, _P, ctypes.POINTER(MbeStats)]),
    "osvmp2_fragment_results": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "osvmp2_profile": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "osvmp2_mbe3_fragments": (ctypes.c_int, [_P, _I32, _D, _D, _I64, _P, _P, _P]),
    "osvmp2_energy_grad": (ctypes.c_int, [_P, _D, _D, ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(MbeStats)]),
    "osvmp2_energy_grad_relaxed": (ctypes.c_int, [_P, _D, _D, _P, _P, _P, _P, ctypes.POINTER(MbeStats), _P]),
    "osvmp2_pair_screening": (ctypes.c_int, [_P, ctypes.POINTER(Screen), _P, _P, _P]),
    "osvmp2_mbe3_energy_screened": (ctypes.c_int, [_P, ctypes.POINTER(Screen), ctypes.c_int, _P, _P,
                                                   ctypes.POINTER(MbeStats)]),
    "osvmp2_weak_results": (ctypes.c_int, [_P, _P, _P, _P]),
    "osvmp2_localize_pm": (ctypes.c_int, [_P, _P, _I32, _I32, _P, _I32, _D, _I32, _P, _P, _P]),
    "osvmp2_precond_noalloc": (ctypes.c_int, [_P, _P, _I32, _D, _P, _P, _P, _P, ctypes.c_char_p, _I32]),
    "osvmp2_generate_B": (ctypes.c_int, [_I32, _I32, _I32, ctypes.c_uint64, _P, _I32, _I32, _P, _P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libosvmp2.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class OSVMP2Error(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} -> {STATUS.get(code, code)}: {msg}")
        self.code = code


def _ptr(x) -> Optional[int]:
    """Device pointer of a torch tensor, host pointer of a numpy array, or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _need_f64_cuda(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")


def default_opts() -> Opts:
    o = Opts()
    lib().osvmp2_default_opts(ctypes.byref(o))
    return o


def kernel_launches() -> int:
    """Kernels launched by libosvmp2 in this process so far."""
    return int(lib().osvmp2_kernel_launches())


def mbe3_fragments(r_occ: np.ndarray, r2_cut: float, r3_cut: float):
    """Host-only fragment enumeration (same rule as osvmp2_mbe3_energy).
    Returns (orbs [n,3] int32, -1 padded; weights [n] int32)."""
    r = np.ascontiguousarray(r_occ, dtype=np.float64)
    n = ctypes.c_int64(0)
    s = lib().osvmp2_mbe3_fragments(_ptr(r), r.shape[0], r2_cut, r3_cut, 0, None, None, ctypes.byref(n))
    if s:
        raise OSVMP2Error("osvmp2_mbe3_fragments", s, "bad arguments")
    orbs = np.empty((n.value, 3), dtype=np.int32)
    w = np.empty(n.value, dtype=np.int32)
    s = lib().osvmp2_mbe3_fragments(_ptr(r), r.shape[0], r2_cut, r3_cut, n.value, _ptr(orbs), _ptr(w),
                                    ctypes.byref(n))
    if s:
        raise OSVMP2Error("osvmp2_mbe3_fragments", s, "bad arguments")
    return orbs, w


def generate_B(n_occ, n_vir, n_aux, seed, env, i0=0, n_i=None, out=None, stream=None):
    """B[i0:i0+n_i] regenerated on the device (torch float64 CUDA tensor)."""
    import torch
    _need_f64_cuda(env, "env")
    n_i = n_occ - i0 if n_i is None else n_i
    if out is None:
        out = torch.empty((n_i, n_vir, n_aux), dtype=torch.float64, device=env.device)
    st = stream if stream is not None else torch.cuda.current_stream(env.device).cuda_stream
    s = lib().osvmp2_generate_B(n_occ, n_vir, n_aux, seed, _ptr(env), i0, n_i, _ptr(out), st)
    if s:
        raise OSVMP2Error("osvmp2_generate_B", s, "launch failed")
    return out


NOALLOC_MAX_M = 256


def precond_noalloc(S, F, tau_s, X, et, r, stream=None) -> None:
    """Allocation-free preconditioner of one pair (osvmp2_precond_noalloc): S, F
    [m, m] float64 CUDA tensors in, X [m, m], et [>= m] float64 and r [>= 1] int32
    CUDA tensors out, preallocated by the caller on the same device.  r receives
    the number of kept directions (0 if S has none above tau_s * max, -1 if an
    eigen-solve failed or met a non-finite value).  Raises TypeError or
    ValueError for tensors of the wrong kind or size (the kernel would otherwise
    write past their end), OSVMP2Error on a non-OK status."""
    import torch
    for t, name in ((S, "S"), (F, "F"), (X, "X"), (et, "et")):
        _need_f64_cuda(t, name)
    if not (isinstance(r, torch.Tensor) and r.is_cuda and r.dtype == torch.int32):
        raise TypeError("r must be an int32 CUDA tensor")
    if S.dim() != 2 or S.shape[0] != S.shape[1]:
        raise ValueError(f"S must be square, got {tuple(S.shape)}")
    m = S.shape[0]
    if tuple(F.shape) != (m, m):
        raise ValueError(f"F must have S's shape {(m, m)}, got {tuple(F.shape)}")
    if tuple(X.shape) != (m, m):
        raise ValueError(f"X must be [{m}, {m}], got {tuple(X.shape)}")
    if et.numel() < m:
        raise ValueError(f"et needs at least {m} entries, got {et.numel()}")
    if r.numel() < 1:
        raise ValueError("r needs one element")
    if len({t.device for t in (S, F, X, et, r)}) != 1:
        raise ValueError("S, F, X, et and r must be on one device")
    st = stream if stream is not None else torch.cuda.current_stream(S.device).cuda_stream
    buf = ctypes.create_string_buffer(256)
    code = lib().osvmp2_precond_noalloc(_ptr(S), _ptr(F), m, tau_s, _ptr(X), _ptr(et), _ptr(r), st, buf, 256)
    if code:
        raise OSVMP2Error("osvmp2_precond_noalloc", code, buf.value.decode())


def _apply_opts(o: Opts, kw) -> None:
    for k, v in kw.items():
        if k == "osv_prec" and isinstance(v, str):
            v = PREC[v]
        if k == "osv_method" and isinstance(v, str):
            v = {"exact": 0, "randomized": 1}[v]
        setattr(o, k, v)


class Context:
    """One osvmp2_ctx on a CUDA device and stream (defaults: current device/stream)."""

    def __init__(self, device: int = 0, stream=None, opts: Optional[Opts] = None, **kw):
        import torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        o = opts or default_opts()
        _apply_opts(o, kw)
        self.opts = o
        h = ctypes.c_void_p()
        s = lib().osvmp2_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(o))
        if s:
            raise OSVMP2Error("osvmp2_create", s, "could not create context")
        self._h = h
        self._keep = ()
        self.n_occ = self.n_vir = self.n_aux = 0

    def set_opts(self, **kw):
        """Change options (e.g. osv_prec="mixed") for the following calls."""
        o = Opts()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(self.opts), ctypes.sizeof(Opts))
        _apply_opts(o, kw)
        self._check("osvmp2_set_opts", lib().osvmp2_set_opts(self._h, ctypes.byref(o)))
        self.opts = o

    def solve_plan(self):
        """Launch shape of the last mixed MBE(3) solve: dict(ctas_per_sm, tiles, tuned, n_keys)."""
        out = (ctypes.c_int32 * 4)()
        self._check("osvmp2_get_solve_plan", lib().osvmp2_get_solve_plan(self._h, out))
        return {"ctas_per_sm": out[0], "tiles": out[1], "tuned": bool(out[2]), "n_keys": out[3]}

    def close(self):
        if getattr(self, "_h", None):
            lib().osvmp2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, fn, code):
        if code:
            raise OSVMP2Error(fn, code, lib().osvmp2_last_error(self._h).decode())

    # ---- A0
    def build_osv(self, f_occ, e_vir, l_osv: float, B=None, env=None, seed: int = 0,
                  r_occ: Optional[np.ndarray] = None, n_aux: Optional[int] = None) -> np.ndarray:
        """OSVs of every orbital.  Device tensors: B [n_occ,n_vir,n_aux] or env [n_occ,n_vir]
        (then B is regenerated from ``seed``), f_occ [n_occ,n_occ], e_vir [n_vir].
        r_occ: host [n_occ,3].  Returns n_osv (numpy int32)."""
        _need_f64_cuda(f_occ, "f_occ")
        _need_f64_cuda(e_vir, "e_vir")
        if B is not None:
            _need_f64_cuda(B, "B")
            n_occ, n_vir, nx = B.shape
        else:
            _need_f64_cuda(env, "env")
            n_occ, n_vir = env.shape
            if n_aux is None:
                raise ValueError("n_aux is required when B is regenerated")
            nx = n_aux
        r = None if r_occ is None else np.ascontiguousarray(r_occ, dtype=np.float64)
        sysd = System(n_occ, n_vir, nx, _ptr(B), seed, _ptr(env), _ptr(f_occ), _ptr(e_vir), _ptr(r))
        n_osv = np.zeros(n_occ, dtype=np.int32)
        self._check("osvmp2_build_osv", lib().osvmp2_build_osv(self._h, ctypes.byref(sysd), l_osv, _ptr(n_osv)))
        self._keep = (B, env, f_occ, e_vir, r)
        self.n_occ, self.n_vir, self.n_aux = n_occ, n_vir, nx
        self.n_osv = n_osv
        return n_osv

    def get_osv(self, i: int):
        import torch
        k = int(self.n_osv[i])
        Q = torch.empty((self.n_vir, k), dtype=torch.float64, device=f"cuda:{self.device}")
        w = torch.empty(k, dtype=torch.float64, device=f"cuda:{self.device}")
        self._check("osvmp2_get_osv", lib().osvmp2_get_osv(self._h, i, _ptr(Q), _ptr(w)))
        return Q, w

    # ---- A1-A3
    def pair_integrals(self, pairs: Sequence[Sequence[int]], prec: str = "fp64"):
        p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self._check("osvmp2_pair_integrals",
                    lib().osvmp2_pair_integrals(self._h, _ptr(p), p.shape[0], PREC[prec]))

    def get_pair_blocks(self, i: int, j: int):
        import torch
        m = int(self.n_osv[i] + (self.n_osv[j] if i != j else 0))
        K, S, F = (torch.empty((m, m), dtype=torch.float64, device=f"cuda:{self.device}") for _ in range(3))
        self._check("osvmp2_get_pair_blocks", lib().osvmp2_get_pair_blocks(self._h, i, j, _ptr(K), _ptr(S), _ptr(F)))
        return K, S, F

    def get_precond(self, i: int, j: int):
        """(X [m, r], e~ [r]) of built pair (i, j)."""
        import torch
        m = int(self.n_osv[i] + (self.n_osv[j] if i != j else 0))
        X = torch.empty((m, m), dtype=torch.float64, device=f"cuda:{self.device}")
        et = torch.empty(m, dtype=torch.float64, device=f"cuda:{self.device}")
        r = ctypes.c_int32(0)
        self._check("osvmp2_get_precond", lib().osvmp2_get_precond(self._h, i, j, _ptr(X), _ptr(et), ctypes.addressof(r)))
        return X[:, :r.value], et[:r.value]

    # ---- A3-A4
    def solve(self, orbs: Sequence[int], prec: str = "fp64"):
        """Returns (E, pair energies [n(n+1)/2] for i<=j in orbs order, iterations)."""
        o = np.ascontiguousarray(np.asarray(orbs, dtype=np.int32))
        n = o.shape[0]
        e = ctypes.c_double(0.0)
        it = ctypes.c_int32(0)
        pe = np.zeros(n * (n + 1) // 2)
        self._check("osvmp2_solve", lib().osvmp2_solve(self._h, _ptr(o), n, PREC[prec], ctypes.addressof(e),
                                                       _ptr(pe), ctypes.addressof(it)))
        return e.value, pe, it.value

    # ---- A5
    def mbe3_energy(self, r2_cut: float, r3_cut: float, prec: str = "fp64"):
        e = ctypes.c_double(0.0)
        st = MbeStats()
        self._check("osvmp2_mbe3_energy", lib().osvmp2_mbe3_energy(self._h, r2_cut, r3_cut, PREC[prec],
                                                                   ctypes.addressof(e), ctypes.byref(st)))
        return e.value, st.as_dict()

    PHASES = ["tii", "eig", "sf", "project", "exchange", "precond", "solve", "mbe_sum", "subsolve", "grad",
              "k_gproj", "k_eig", "k_fragsolve", "sigma", "weak", "screen", "localize", "relax", "spare18",
              "spare19"]

    # ---- occupied-orbital localization (Algorithm 2)
    def localize_pm(self, C, atom_ao, l_loc: float = 1e-3, max_sweeps: int = 100):
        """Pipek-Mezey localization of the columns of C (float64 CUDA [n_ao, n_occ]);
        atom_ao: AO offsets of the atoms.  Returns (U [n_occ, n_occ] CUDA tensor, L, sweeps)."""
        import torch
        _need_f64_cuda(C, "C")
        n_ao, n = C.shape
        ao = np.ascontiguousarray(np.asarray(atom_ao, dtype=np.int32))
        U = torch.empty((n, n), dtype=torch.float64, device=C.device)
        L = ctypes.c_double(0.0)
        sw = ctypes.c_int32(0)
        self._check("osvmp2_localize_pm",
                    lib().osvmp2_localize_pm(self._h, _ptr(C), n_ao, n, _ptr(ao), ao.shape[0] - 1, l_loc, max_sweeps,
                                             _ptr(U), ctypes.addressof(L), ctypes.addressof(sw)))
        return U, L.value, sw.value

    # ---- A5 with the paper's cluster selection
    def pair_screening(self, screen: Optional[Screen] = None):
        """(s2b [n,n], class [n,n] (2 close, 1 weak, 0 distant), counts (close, weak, distant))."""
        sc = screen or Screen()
        n = self.n_occ
        s2b = np.zeros((n, n))
        cls = np.zeros((n, n), dtype=np.int32)
        cnt = np.zeros(3, dtype=np.int64)
        self._check("osvmp2_pair_screening",
                    lib().osvmp2_pair_screening(self._h, ctypes.byref(sc), _ptr(s2b), _ptr(cls), _ptr(cnt)))
        return s2b, cls, tuple(int(x) for x in cnt)

    def mbe3_energy_screened(self, prec: str = "fp64", screen: Optional[Screen] = None):
        """(E, E_weak, stats) of the MBE(3) energy over the s2b/s3b-selected clusters plus weak pairs."""
        sc = screen or Screen()
        e = ctypes.c_double(0.0)
        ew = ctypes.c_double(0.0)
        st = MbeStats()
        self._check("osvmp2_mbe3_energy_screened",
                    lib().osvmp2_mbe3_energy_screened(self._h, ctypes.byref(sc), PREC[prec], ctypes.addressof(e),
                                                      ctypes.addressof(ew), ctypes.byref(st)))
        return e.value, ew.value, st.as_dict()

    def weak_results(self):
        """(pairs [n,2] int32, energies [n]) of the last screened call."""
        n = ctypes.c_int64(0)
        self._check("osvmp2_weak_results", lib().osvmp2_weak_results(self._h, ctypes.byref(n), None, None))
        pairs = np.empty((n.value, 2), dtype=np.int32)
        e = np.empty(n.value)
        self._check("osvmp2_weak_results",
                    lib().osvmp2_weak_results(self._h, ctypes.byref(n), _ptr(pairs), _ptr(e)))
        return pairs, e

    def profile(self, reset: bool = False):
        """Per-phase {name: (ms, flops, bytes, calls)} accumulated since the last reset."""
        n = len(self.PHASES)
        ms, fl, by = np.zeros(n), np.zeros(n), np.zeros(n)
        calls = np.zeros(n, dtype=np.int64)
        self._check("osvmp2_profile", lib().osvmp2_profile(self._h, _ptr(ms), _ptr(fl), _ptr(by), _ptr(calls), int(reset)))
        return {self.PHASES[k]: (float(ms[k]), float(fl[k]), float(by[k]), int(calls[k])) for k in range(n) if calls[k]}

    def fragment_results(self):
        n = ctypes.c_int64(0)
        self._check("osvmp2_fragment_results", lib().osvmp2_fragment_results(self._h, ctypes.byref(n), None, None, None))
        orbs = np.empty((n.value, 3), dtype=np.int32)
        w = np.empty(n.value, dtype=np.int32)
        e = np.empty(n.value)
        self._check("osvmp2_fragment_results",
                    lib().osvmp2_fragment_results(self._h, ctypes.byref(n), _ptr(orbs), _ptr(w), _ptr(e)))
        return orbs, w, e

    # ---- A6
    def energy_grad(self, r2_cut: float, r3_cut: float, prec: str = "fp64", want_dB: bool = True):
        import torch
        dev = f"cuda:{self.device}"
        dB = torch.empty((self.n_occ, self.n_vir, self.n_aux), dtype=torch.float64, device=dev) if want_dB else None
        df = torch.empty((self.n_occ, self.n_occ), dtype=torch.float64, device=dev)
        de = torch.empty(self.n_vir, dtype=torch.float64, device=dev)
        e = ctypes.c_double(0.0)
        st = MbeStats()
        self._check("osvmp2_energy_grad",
                    lib().osvmp2_energy_grad(self._h, r2_cut, r3_cut, PREC[prec], ctypes.addressof(e), _ptr(dB),
                                             _ptr(df), _ptr(de), ctypes.byref(st)))
        return e.value, dB, df, de, st.as_dict()

    def energy_grad_relaxed(self, r2_cut: float, r3_cut: float, want_dB: bool = True):
        """energy_grad (FP64 form) plus the response of the OSVs to T_ii, counts held
        fixed.  Returns (E, dB, df, de, stats, smallest eigenvalue gap at the OSV cut)."""
        import torch
        dev = f"cuda:{self.device}"
        dB = torch.empty((self.n_occ, self.n_vir, self.n_aux), dtype=torch.float64, device=dev) if want_dB else None
        df = torch.empty((self.n_occ, self.n_occ), dtype=torch.float64, device=dev)
        de = torch.empty(self.n_vir, dtype=torch.float64, device=dev)
        e = ctypes.c_double(0.0)
        gap = ctypes.c_double(0.0)
        st = MbeStats()
        self._check("osvmp2_energy_grad_relaxed",
                    lib().osvmp2_energy_grad_relaxed(self._h, r2_cut, r3_cut, ctypes.addressof(e), _ptr(dB), _ptr(df),
                                                     _ptr(de), ctypes.byref(st), ctypes.addressof(gap)))
        return e.value, dB, df, de, st.as_dict(), gap.value


def mbe3_energy_function():
    """torch.autograd.Function around osvmp2_energy_grad / osvmp2_energy_grad_relaxed.

    forward(ctx_obj, B, f_occ, e_vir, r_occ, r2, r3, prec, l_osv, relaxed) -> E (0-dim float64 tensor)
    backward: dE/dB, dE/df_occ (symmetrised) and dE/de_vir from the adjoint kernels, each
    scaled by the incoming gradient; with the OSVs held fixed, or with relaxed=True (FP64
    form) including their response to T_ii at fixed OSV counts.
    """
    import torch

    class _MBE3Energy(torch.autograd.Function):
        @staticmethod
        def forward(fctx, ctx_obj, B, f_occ, e_vir, r_occ, r2, r3, prec="fp64", l_osv=1e-4, relaxed=False):
            ctx_obj.build_osv(f_occ, e_vir, l_osv, B=B, r_occ=r_occ)
            if relaxed:
                if prec != "fp64":
                    raise ValueError("the relaxed gradient runs in the FP64 form only")
                E, dB, df, de, _, _ = ctx_obj.energy_grad_relaxed(r2, r3, want_dB=True)
            else:
                E, dB, df, de, _ = ctx_obj.energy_grad(r2, r3, prec, want_dB=True)
            fctx.save_for_backward(dB, df, de)
            return torch.tensor(E, dtype=torch.float64, device=B.device)

        @staticmethod
        def backward(fctx, g):
            dB, df, de = fctx.saved_tensors
            return None, g * dB, g * df, g * de, None, None, None, None, None, None

    return _MBE3Energy
