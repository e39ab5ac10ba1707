"""ctypes binding of libafqmc_kp.so (argument marshalling only).

Every operation runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream.  If the library is missing or cannot be loaded
the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libafqmc_kp.so")

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "singular walker overlap",
          5: "timeout", 6: "unsupported"}
FP64, MIXED = 0, 1
PRECISIONS = {"fp64": FP64, "mixed": MIXED}

# Entry points declared in include/afqmc_kp.h, with their ctypes signatures.
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "afqmc_kp_create": [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)],
    "afqmc_kp_destroy": [_VP],
    "afqmc_dense_create": [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)],
    "afqmc_kp_set_one_body": [_VP, _VP, _VP],
    "afqmc_kp_force_bias": [_VP, _VP, _VP, _VP],
    "afqmc_kp_propagate": [_VP, _VP, _VP, _VP, _VP, _I, _VP],
    "afqmc_kp_orthonormalise": [_VP, _VP, _VP, _VP],
    "afqmc_kp_step": [_VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _VP],
    "afqmc_kp_local_energy": [_VP, _VP, _VP, _VP],
    "afqmc_kp_local_energy_backward": [_VP, _VP, _VP, _VP, _VP, _VP],
    "afqmc_kp_last_error": [_VP, _VP, ctypes.POINTER(_I)],
    "afqmc_kp_wait_selftest": [_VP, _I, ctypes.c_longlong, _VP],
    "afqmc_kp_memory_bytes": [_VP, ctypes.POINTER(ctypes.c_size_t)],
    "afqmc_kp_launch_count": [_VP, ctypes.POINTER(_I)],
    "afqmc_kp_profile": [_VP, _I],
    "afqmc_kp_stage_times": [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)],
    "afqmc_status_string": [_I],
    "afqmc_last_message": [],
    "afqmc_orthonormalise_noalloc": [_VP, _I, _I, _I, _VP],
    "afqmc_kp_group_create": [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP)],
    "afqmc_kp_group_destroy": [_VP],
    "afqmc_kp_group_step": [_VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _VP],
    "afqmc_kp_group_block": [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _I, _I, ctypes.c_ulonglong, _VP, _VP],
    "afqmc_kp_group_launch_count": [_VP, ctypes.POINTER(_I)],
    "afqmc_kp_group_set_shared": [_VP, _I],
    "afqmc_kp_group_shared": [_VP, ctypes.POINTER(_I)],
    "afqmc_kp_gemm_tuning": [_VP, _VP, _VP, _VP, ctypes.POINTER(_I)],
    "afqmc_kp_gemm_form": [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)],
    "afqmc_kp_set_gemm_form": [_VP, _I, _I],
    "afqmc_philox4x32_10": [_VP, ctypes.c_ulonglong, _VP, ctypes.c_size_t, _VP],
    "afqmc_kp_fields": [_VP, ctypes.c_ulonglong, _VP, _VP, _VP],
    "afqmc_kp_comb": [_VP, _VP, _VP, ctypes.c_ulonglong, _VP, _VP, _VP],
    "afqmc_kp_block": [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _I, _I, ctypes.c_ulonglong, _VP, _VP, _VP],
}


class Desc(ctypes.Structure):
    _fields_ = [("kgrid", ctypes.c_int * 3), ("M", _I), ("nocc", _I), ("nchol", _I), ("nwalkers", _I),
                ("dt", _D), ("taylor_order", _I), ("prec", _I), ("workspace_cap_bytes", ctypes.c_size_t)]


class DenseDesc(ctypes.Structure):
    _fields_ = [("M", _I), ("nocc", _I), ("nchol", _I), ("nwalkers", _I), ("dt", _D), ("taylor_order", _I),
                ("prec", _I), ("hermitian", _I), ("workspace_cap_bytes", ctypes.c_size_t)]


class AfqmcError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("afqmc_status_string", "afqmc_last_message") else ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        msg = _lib.afqmc_last_message().decode() if _lib is not None else ""
        raise AfqmcError(status, where + (f" [{msg}]" if msg else ""))


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: torch.Tensor, dtype, shape, name) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.is_complex() and (t.is_conj() or t.is_neg()):
        # a lazy conjugate or negative view shares the unconjugated storage: its data pointer
        # would hand the library the wrong values
        raise ValueError(f"{name} is a lazy conjugate/negative view: pass t.resolve_conj().resolve_neg()")
    return t.data_ptr()


def _as_c128(a) -> torch.Tensor:
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))
    return a.to(torch.complex128).contiguous()


class KPointAFQMC:
    """One k-point Hamiltonian + trial on the current CUDA device (a library handle)."""

    def __init__(self, grid, L, h1, trial, nwalkers: int, dt: float, taylor_order: int = 6,
                 precision: str = "fp64", workspace_cap_bytes: int = 0, stream=None):
        lib = load_library()
        self.lib = lib
        L = _as_c128(L)
        h1 = _as_c128(h1)
        trial = _as_c128(trial)
        nk, _, G, M, _ = L.shape
        n = trial.shape[2]
        self.grid = tuple(int(g) for g in grid)
        if int(np.prod(self.grid)) != nk:
            raise ValueError("grid does not match L")
        self.nk, self.M, self.n, self.G, self.W = nk, M, n, G, int(nwalkers)
        self.NM, self.N = nk * M, nk * n
        self.dt = float(dt)
        self.precision = precision
        d = Desc()
        d.kgrid[:] = list(self.grid)
        d.M, d.nocc, d.nchol, d.nwalkers = M, n, G, self.W
        d.dt = self.dt
        d.taylor_order = int(taylor_order)
        d.prec = PRECISIONS[precision]
        d.workspace_cap_bytes = int(workspace_cap_bytes)
        # host inputs are passed as host pointers (the library copies them)
        keep = [t if t.is_cuda else t.contiguous() for t in (L, h1, trial)]
        handle = ctypes.c_void_p()
        _check(lib.afqmc_kp_create(ctypes.byref(d), keep[0].data_ptr(), keep[1].data_ptr(), keep[2].data_ptr(),
                                   _stream(stream), ctypes.byref(handle)), "afqmc_kp_create")
        self.handle = handle
        self.h1 = h1.cuda() if not h1.is_cuda else h1

    # shapes -------------------------------------------------------------
    @property
    def phi_shape(self):
        return (self.W, 2, self.NM, self.N)

    @property
    def field_shape(self):
        return (self.W, 2, self.nk, self.G)

    def close(self):
        if getattr(self, "handle", None):
            _check(self.lib.afqmc_kp_destroy(self.handle), "afqmc_kp_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # calls --------------------------------------------------------------
    def set_one_body(self, h1: torch.Tensor, stream=None):
        p = _ptr(h1, torch.complex128, (self.nk, self.M, self.M), "h1")
        _check(self.lib.afqmc_kp_set_one_body(self.handle, p, _stream(stream)), "afqmc_kp_set_one_body")

    def force_bias(self, phi: torch.Tensor, xbar: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if xbar is None:
            xbar = torch.empty((self.W, 2, self.nk, self.G), dtype=torch.complex128, device=phi.device)
        _check(self.lib.afqmc_kp_force_bias(self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
                                            _ptr(xbar, torch.complex128, xbar.shape, "xbar"), _stream(stream)),
               "afqmc_kp_force_bias")
        return xbar

    def propagate(self, phi, x, weight, logdet=None, do_qr=False, stream=None):
        lp = 0 if logdet is None else _ptr(logdet, torch.complex128, (self.W, 2), "logdet")
        _check(self.lib.afqmc_kp_propagate(self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
                                           _ptr(x, torch.float64, self.field_shape, "x"),
                                           _ptr(weight, torch.float64, (self.W,), "weight"), lp,
                                           1 if do_qr else 0, _stream(stream)), "afqmc_kp_propagate")

    def step(self, phi, x, weight, eloc=None, logdet=None, do_qr=False, reuse=True, energy=True,
             stream=None) -> Optional[torch.Tensor]:
        """Propagate every walker one step and return the local energy of the new walkers
        (energy=False: a propagation-only step, returns None)."""
        if eloc is None and energy:
            eloc = torch.empty((self.W, 3), dtype=torch.complex128, device=phi.device)
        ep = _ptr(eloc, torch.complex128, (self.W, 3), "eloc") if energy else 0
        lp = 0 if logdet is None else _ptr(logdet, torch.complex128, (self.W, 2), "logdet")
        _check(self.lib.afqmc_kp_step(self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
                                      _ptr(x, torch.float64, self.field_shape, "x"),
                                      _ptr(weight, torch.float64, (self.W,), "weight"), ep, lp,
                                      1 if do_qr else 0, 1 if reuse else 0, _stream(stream)), "afqmc_kp_step")
        return eloc if energy else None

    def orthonormalise(self, phi, logdet=None, stream=None):
        lp = 0 if logdet is None else _ptr(logdet, torch.complex128, (self.W, 2), "logdet")
        _check(self.lib.afqmc_kp_orthonormalise(self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
                                                lp, _stream(stream)), "afqmc_kp_orthonormalise")

    def local_energy(self, phi, eloc=None, stream=None) -> torch.Tensor:
        if eloc is None:
            eloc = torch.empty((self.W, 3), dtype=torch.complex128, device=phi.device)
        _check(self.lib.afqmc_kp_local_energy(self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
                                              _ptr(eloc, torch.complex128, (self.W, 3), "eloc"), _stream(stream)),
               "afqmc_kp_local_energy")
        return eloc

    def local_energy_backward(self, phi, grad_e, want_phi=True, want_h1=True, stream=None
                              ) -> Tuple[Optional[torch.Tensor], Optional[torch.Tensor]]:
        gphi = torch.empty(self.phi_shape, dtype=torch.complex128, device=phi.device) if want_phi else None
        gh1 = torch.empty((self.nk, self.M, self.M), dtype=torch.complex128, device=phi.device) if want_h1 else None
        _check(self.lib.afqmc_kp_local_energy_backward(
            self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
            _ptr(grad_e, torch.complex128, (self.W, 3), "grad_e"),
            0 if gphi is None else gphi.data_ptr(), 0 if gh1 is None else gh1.data_ptr(), _stream(stream)),
            "afqmc_kp_local_energy_backward")
        return gphi, gh1

    def fields(self, counter: torch.Tensor, seed: int, x: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Standard normal fields x[W][2][Nk][G] from Philox4x32-10 at (seed, counter); advances the counter."""
        if x is None:
            x = torch.empty(self.field_shape, dtype=torch.float64, device=counter.device)
        _check(self.lib.afqmc_kp_fields(self.handle, int(seed) & (2**64 - 1),
                                        _ptr(counter, torch.int64, (1,), "counter"),
                                        _ptr(x, torch.float64, self.field_shape, "x"), _stream(stream)),
               "afqmc_kp_fields")
        return x

    def comb(self, phi, weight, counter: torch.Tensor, seed: int, idx: Optional[torch.Tensor] = None, stream=None):
        """Comb population control in place on (phi, weight); returns the selected old walker per slot."""
        if idx is None:
            idx = torch.empty((self.W,), dtype=torch.int32, device=phi.device)
        _check(self.lib.afqmc_kp_comb(self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
                                      _ptr(weight, torch.float64, (self.W,), "weight"), int(seed) & (2**64 - 1),
                                      _ptr(counter, torch.int64, (1,), "counter"),
                                      _ptr(idx, torch.int32, (self.W,), "idx"), _stream(stream)), "afqmc_kp_comb")
        return idx

    def block(self, phi, weight, x, eloc_hist, counter: torch.Tensor, seed: int, nsteps: Optional[int] = None,
              qr_period: int = 5, energy_period: int = 1, weight_hist=None, logdet=None, comb=True, reuse=False,
              idx=None, stream=None):
        """One device-driven block (afqmc_kp_block): nsteps steps (default: one per eloc_hist row times
        energy_period), energy every energy_period steps and after the last, then the comb."""
        nmeas = int(eloc_hist.shape[0])
        if nsteps is None:
            nsteps = nmeas * int(energy_period)
        if nmeas != -(-int(nsteps) // int(energy_period)):
            raise ValueError("eloc_hist needs ceil(nsteps / energy_period) rows")
        eh = _ptr(eloc_hist, torch.complex128, (nmeas, self.W, 3), "eloc_hist")
        wh = 0 if weight_hist is None else _ptr(weight_hist, torch.float64, (nsteps, self.W), "weight_hist")
        lp = 0 if logdet is None else _ptr(logdet, torch.complex128, (self.W, 2), "logdet")
        ip = 0 if idx is None else _ptr(idx, torch.int32, (self.W,), "idx")
        _check(self.lib.afqmc_kp_block(self.handle, _ptr(phi, torch.complex128, self.phi_shape, "phi"),
                                       _ptr(weight, torch.float64, (self.W,), "weight"),
                                       _ptr(x, torch.float64, self.field_shape, "x"), eh, wh, lp, int(nsteps),
                                       int(qr_period), int(energy_period), 1 if reuse else 0, 1 if comb else 0,
                                       int(seed) & (2**64 - 1), _ptr(counter, torch.int64, (1,), "counter"), ip,
                                       _stream(stream)), "afqmc_kp_block")

    def last_error(self, stream=None) -> Tuple[int, int]:
        n = ctypes.c_int(0)
        s = self.lib.afqmc_kp_last_error(self.handle, _stream(stream), ctypes.byref(n))
        return s, n.value

    def wait_selftest(self, arrive: bool, limit_cycles: int, stream=None):
        """One bounded mbarrier wait on the device (afqmc_kp_wait_selftest); without the
        arrival it gives up after limit_cycles and records a time-out in the sticky flags."""
        _check(self.lib.afqmc_kp_wait_selftest(self.handle, 1 if arrive else 0, int(limit_cycles), _stream(stream)),
               "afqmc_kp_wait_selftest")

    def memory_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check(self.lib.afqmc_kp_memory_bytes(self.handle, ctypes.byref(b)), "afqmc_kp_memory_bytes")
        return b.value

    STAGES = ("green", "force_bias", "vhs", "taylor", "weight", "qr", "energy", "exchange", "backward", "onebody",
              "adjoint_gemm")

    def profile(self, enable: bool = True):
        _check(self.lib.afqmc_kp_profile(self.handle, 1 if enable else 0), "afqmc_kp_profile")

    def stage_times(self):
        """{stage: (milliseconds, intervals)} recorded since the last read (synchronises)."""
        ms = (ctypes.c_double * len(self.STAGES))()
        cnt = (ctypes.c_int * len(self.STAGES))()
        _check(self.lib.afqmc_kp_stage_times(self.handle, ms, cnt), "afqmc_kp_stage_times")
        return {s: (ms[i], cnt[i]) for i, s in enumerate(self.STAGES)}

    def launch_count(self) -> int:
        n = ctypes.c_int(0)
        _check(self.lib.afqmc_kp_launch_count(self.handle, ctypes.byref(n)), "afqmc_kp_launch_count")
        return n.value

    GEMMS = ("green", "force_bias", "vhs", "taylor", "exchange", "adjoint", "gram", "apply_r")

    def gemm_tuning(self):
        """{gemm: {"ring_depth", "ms_2_stages", "ms_3_stages"}} chosen at create (empty for FP64)."""
        n = len(self.GEMMS)
        depth, ms2, ms3 = (ctypes.c_int * n)(), (ctypes.c_double * n)(), (ctypes.c_double * n)()
        cnt = ctypes.c_int(0)
        _check(self.lib.afqmc_kp_gemm_tuning(self.handle, depth, ms2, ms3, ctypes.byref(cnt)),
               "afqmc_kp_gemm_tuning")
        out = {self.GEMMS[i]: {"ring_depth": depth[i], "ms_2_stages": ms2[i], "ms_3_stages": ms3[i]}
               for i in range(cnt.value)}
        for name in out:
            pair, ms = self.gemm_form(name)
            out[name]["cta_pair"] = pair
            if ms != 0.0:
                out[name]["ms_cta_pair"] = ms
        return out

    def gemm_form(self, gemm: str):
        """(pair, ms_pair): whether the GEMM runs in the CTA-pair form, and its ms at create."""
        pair, ms = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(self.lib.afqmc_kp_gemm_form(self.handle, self.GEMMS.index(gemm), ctypes.byref(pair), ctypes.byref(ms)),
               "afqmc_kp_gemm_form")
        return bool(pair.value), ms.value

    def set_gemm_form(self, gemm: str, pair: bool):
        _check(self.lib.afqmc_kp_set_gemm_form(self.handle, self.GEMMS.index(gemm), 1 if pair else 0),
               "afqmc_kp_set_gemm_form")


def _ptr_array(ptrs):
    """Host array of device pointers (kept alive by the caller for the call)."""
    return (_VP * len(ptrs))(*ptrs)


class DenseAFQMC(KPointAFQMC):
    """A standard-representation system (afqmc_dense_create): M orbitals, vectors L[G][M][M].
    It is a single-k-point handle with G' Hermitian vectors; fields and force biases use the
    layout [W][2][1][G'] (plane 0: the + fields, then for general vectors the - fields)."""

    def __init__(self, L, h1, trial, nwalkers: int, dt: float, taylor_order: int = 6, precision: str = "fp64",
                 hermitian: bool = False, workspace_cap_bytes: int = 0, stream=None):
        lib = load_library()
        self.lib = lib
        L = _as_c128(L)
        h1 = _as_c128(h1)
        trial = _as_c128(trial)
        G, M, _ = L.shape
        n = trial.shape[1]
        self.grid = (1, 1, 1)
        self.hermitian = bool(hermitian)
        self.nchol_dense = G
        self.nk, self.M, self.n, self.W = 1, M, n, int(nwalkers)
        self.G = G if self.hermitian else 2 * G
        self.NM, self.N = M, n
        self.dt = float(dt)
        self.precision = precision
        d = DenseDesc()
        d.M, d.nocc, d.nchol, d.nwalkers = M, n, G, self.W
        d.dt = self.dt
        d.taylor_order = int(taylor_order)
        d.prec = PRECISIONS[precision]
        d.hermitian = 1 if self.hermitian else 0
        d.workspace_cap_bytes = int(workspace_cap_bytes)
        keep = [t if t.is_cuda else t.contiguous() for t in (L, h1, trial)]
        handle = ctypes.c_void_p()
        _check(lib.afqmc_dense_create(ctypes.byref(d), keep[0].data_ptr(), keep[1].data_ptr(), keep[2].data_ptr(),
                                      _stream(stream), ctypes.byref(handle)), "afqmc_dense_create")
        self.handle = handle
        h1d = h1.reshape(1, M, M)
        self.h1 = h1d.cuda() if not h1d.is_cuda else h1d


class KPointGroup:
    """Several KPointAFQMC systems advanced together, one CUDA stream per member.  Groups of up
    to 8 mixed systems of one Taylor order can share GEMM launches (`shared`): PER_MEMBER (0),
    SHARED_ALL (1, every GEMM kind one launch over all members' tiles) or SHARED_TAYLOR (2, the
    Taylor-term GEMMs only; the default where allowed)."""

    PER_MEMBER, SHARED_ALL, SHARED_TAYLOR = 0, 1, 2

    def __init__(self, systems):
        self.lib = load_library()
        self.systems = list(systems)
        arr = _ptr_array([s.handle.value for s in self.systems])
        g = ctypes.c_void_p()
        _check(self.lib.afqmc_kp_group_create(ctypes.cast(arr, ctypes.POINTER(_VP)), len(self.systems),
                                              ctypes.byref(g)), "afqmc_kp_group_create")
        self.group = g

    def close(self):
        if getattr(self, "group", None):
            _check(self.lib.afqmc_kp_group_destroy(self.group), "afqmc_kp_group_destroy")
            self.group = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, ts, dtype, shapes, name, optional=False):
        if ts is None:
            if optional:
                return None
            raise ValueError(f"{name} is required")
        if len(ts) != len(self.systems):
            raise ValueError(f"{name}: one entry per member")
        return _ptr_array([0 if (t is None and optional) else _ptr(t, dtype, shp, f"{name}[{i}]")
                           for i, (t, shp) in enumerate(zip(ts, shapes))])

    def step(self, phis, xs, weights, elocs=None, logdets=None, do_qr=False, reuse=True, stream=None):
        S = self.systems
        pa = self._arr(phis, torch.complex128, [s.phi_shape for s in S], "phi")
        xa = self._arr(xs, torch.float64, [s.field_shape for s in S], "x")
        wa = self._arr(weights, torch.float64, [(s.W,) for s in S], "weight")
        ea = self._arr(elocs, torch.complex128, [(s.W, 3) for s in S], "eloc", optional=True)
        la = self._arr(logdets, torch.complex128, [(s.W, 2) for s in S], "logdet", optional=True)
        _check(self.lib.afqmc_kp_group_step(self.group, pa, xa, wa, ea, la, 1 if do_qr else 0, 1 if reuse else 0,
                                            _stream(stream)), "afqmc_kp_group_step")

    def block(self, phis, weights, xs, eloc_hists, counters, seed: int, nsteps: int, qr_period: int = 5,
              energy_period: int = 1, weight_hists=None, logdets=None, comb=True, reuse=False, stream=None):
        S = self.systems
        nmeas = -(-int(nsteps) // int(energy_period))
        pa = self._arr(phis, torch.complex128, [s.phi_shape for s in S], "phi")
        wa = self._arr(weights, torch.float64, [(s.W,) for s in S], "weight")
        xa = self._arr(xs, torch.float64, [s.field_shape for s in S], "x")
        ea = self._arr(eloc_hists, torch.complex128, [(nmeas, s.W, 3) for s in S], "eloc_hist")
        ha = self._arr(weight_hists, torch.float64, [(nsteps, s.W) for s in S], "weight_hist", optional=True)
        la = self._arr(logdets, torch.complex128, [(s.W, 2) for s in S], "logdet", optional=True)
        ca = self._arr(counters, torch.int64, [(1,) for _ in S], "counter")
        _check(self.lib.afqmc_kp_group_block(self.group, pa, wa, xa, ea, ha, la, int(nsteps), int(qr_period),
                                             int(energy_period), 1 if reuse else 0, 1 if comb else 0,
                                             int(seed) & (2**64 - 1), ca, _stream(stream)), "afqmc_kp_group_block")

    def launch_count(self) -> int:
        n = ctypes.c_int(0)
        _check(self.lib.afqmc_kp_group_launch_count(self.group, ctypes.byref(n)), "afqmc_kp_group_launch_count")
        return n.value

    @property
    def shared(self) -> int:
        n = ctypes.c_int(0)
        _check(self.lib.afqmc_kp_group_shared(self.group, ctypes.byref(n)), "afqmc_kp_group_shared")
        return n.value

    @shared.setter
    def shared(self, mode: int):
        _check(self.lib.afqmc_kp_group_set_shared(self.group, int(mode)), "afqmc_kp_group_set_shared")


def philox4x32_10(ctr: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Raw Philox4x32-10 words of device counters ctr[n][4] (int32 storage of uint32 values)."""
    lib = load_library()
    n = int(ctr.shape[0])
    out = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    _check(lib.afqmc_philox4x32_10(_ptr(ctr, torch.int32, (n, 4), "ctr"), int(seed) & (2**64 - 1),
                                   out.data_ptr(), n, _stream(stream)), "afqmc_philox4x32_10")
    return out


class LocalEnergy(torch.autograd.Function):
    """E_L parts (W, 3) as a differentiable function of the walkers and of h[k].

    Forward installs h1 in the handle (afqmc_kp_set_one_body) and evaluates the
    local energy; backward calls the library's adjoint kernels.
    """

    @staticmethod
    def forward(ctx, phi, h1, sys: KPointAFQMC):
        sys.set_one_body(h1.detach().contiguous())
        ctx.sys = sys
        ctx.save_for_backward(phi.detach())
        return sys.local_energy(phi.detach().contiguous())

    @staticmethod
    def backward(ctx, grad_e):
        (phi,) = ctx.saved_tensors
        sys = ctx.sys
        grad_e = grad_e.resolve_conj().resolve_neg().contiguous()
        gphi, gh1 = sys.local_energy_backward(phi, grad_e, want_phi=ctx.needs_input_grad[0],
                                              want_h1=ctx.needs_input_grad[1])
        return gphi, gh1, None
