"""Thin ctypes binding of the C ABI in include/tdks.h (argument marshalling only).

Device buffers are torch tensors on the current CUDA device: orbital blocks are
complex128 [n_orb, n_int], quadrature fields float64 [n_elem, nq^3].  Work runs
on torch's current stream.  If libtdks.so is missing this module raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdks.so")

# contraction arithmetic (tdks_prec): FP64; FP32; DF64 double-float (FP64-level,
# on the FP32 pipe); BF16 = bfloat16 operands with FP32 sums (accuracy study only);
# MIXED = double-float Lanczos products until the a-posteriori estimate falls to
# relax * tol, FP32 after (tdks_set_mixed)
FP64, FP32, DF64, BF16, MIXED = 0, 1, 2, 3, 4
PRECOND_FDM, PRECOND_JACOBI = 0, 1
NUC_KIND = {"none": 0, "soft": 1, "erf": 2, "bare": 3, "harmonic": 4}
_dp = C.POINTER(C.c_double)


class MeshDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("X", _dp), ("Y", _dp),
                ("Z", _dp), ("p", C.c_int), ("nq", C.c_int)]


class SystemDesc(C.Structure):
    _fields_ = [("n_orb", C.c_int), ("occ", _dp), ("n_nuc", C.c_int), ("R", _dp), ("Z", _dp),
                ("nuc_kind", C.c_int), ("nuc_param", C.c_double), ("hartree", C.c_int),
                ("xc", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("k_half_max", C.c_int), ("k_full_max", C.c_int), ("applies", C.c_int64),
                ("substeps", C.c_int), ("cg_iters", C.c_int * 3), ("dipole", C.c_double * 3)]

    def as_dict(self):
        return {"k_half_max": self.k_half_max, "k_full_max": self.k_full_max,
                "applies": int(self.applies), "substeps": self.substeps,
                "cg_iters": list(self.cg_iters)[:2], "dipole": list(self.dipole)}


class Counters(C.Structure):
    _fields_ = [("launches", C.c_int64), ("apply_launches", C.c_int64),
                ("apply_elem_orb", C.c_int64), ("apply_ms", C.c_double), ("cg_iters", C.c_int64),
                ("apply_launches_fp32", C.c_int64), ("state_reads", C.c_int64)]


class TDKSError(RuntimeError):
    pass


class TileChoice(C.Structure):
    _fields_ = [("p", C.c_int), ("n_orb", C.c_int), ("elems_per_cta", C.c_int),
                ("orbs_per_item", C.c_int), ("ms", C.c_double)]


_lib = None


def lib():
    """Load libtdks.so (built by paper_1810_13130_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise TDKSError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    v, p, i, d, i64 = C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int64
    sig = {
        "tdks_create": [C.POINTER(MeshDesc), C.POINTER(SystemDesc), v, C.POINTER(C.c_void_p)],
        "tdks_destroy": [v],
        "tdks_set_stream": [v, v],
        "tdks_sizes": [v, C.POINTER(i64), C.POINTER(i64), C.POINTER(i)],
        "tdks_set_cg": [v, d, i, i],
        "tdks_set_potential": [v, p],
        "tdks_nuclear_potential": [v, p],
        "tdks_apply_H": [v, p, p, i, i],
        "tdks_density": [v, p, i, p],
        "tdks_dipole": [v, p, _dp],
        "tdks_hartree": [v, p, p, C.POINTER(i)],
        "tdks_xc": [v, p, p],
        "tdks_expm": [v, p, p, i, d, d, i, i, C.POINTER(i)],
        "tdks_kick": [v, p, i, d, _dp],
        "tdks_init_propagation": [v, p, i, _dp],
        "tdks_magnus_step": [v, p, i, d, _dp, _dp, d, i, i, C.POINTER(Stats)],
        "tdks_propagate_host": [v, p, p, i, i, i, d, p, d, i, i, p],
        "tdks_set_timing": [v, i],
        "tdks_get_counters": [v, C.POINTER(Counters), i],
        "tdks_fma_probe": [i, i, i, i, v, _dp, _dp],
        "tdks_contraction_probe": [i, i, _dp, p, p, i64, i, v, _dp],
        "tdks_last_error": [v],
        "tdks_status_string": [i],
        "tdks_dipole_noalloc": [p, i, i, i, _dp, _dp, _dp, i, v, _dp],
        "tdks_objective_forward": [v, p, i, i, d, _dp, _dp, _dp, i, d, i, i, _dp, _dp],
        "tdks_objective_backward": [v, i, _dp],
        "tdks_set_kb": [v, i, _dp, d, d, _dp, i],
        "tdks_set_lanczos": [v, i],
        "tdks_set_apply_tile": [v, i],
        "tdks_set_f32_stages": [v, C.c_uint],
        "tdks_set_mixed": [v, d],
        "tdks_set_device_loop": [v, i],
        "tdks_magnus_step_sc": [v, p, i, d, _dp, d, i, i, d, i, C.POINTER(Stats), C.POINTER(i)],
        "tdks_apply_H_gll": [v, p, p, p, i],
        "tdks_nuclear_potential_nodes": [v, p],
        "tdks_spectrum": [_dp, i, d, d, _dp, d, _dp, i, _dp, _dp],
        "tdks_kb_info": [v, C.POINTER(i), _dp, C.POINTER(i64), C.POINTER(i64)],
        "tdks_batch_create": [i, p, p, _dp, i, d, i, C.POINTER(C.c_void_p)],
        "tdks_batch_destroy": [v],
        "tdks_batch_stream": [v],
        "tdks_batch_sizes": [v, i, C.POINTER(i64), C.POINTER(i64), C.POINTER(i), C.POINTER(i)],
        "tdks_batch_set_orbitals": [v, i, p],
        "tdks_batch_get_orbitals": [v, i, p],
        "tdks_batch_kick": [v, _dp, _dp],
        "tdks_batch_init": [v, _dp],
        "tdks_batch_tune": [v, i, p, i, C.POINTER(i)],
        "tdks_batch_tune_kmax": [v, i, i64, C.POINTER(i)],
        "tdks_batch_set_kb": [v, i, i, _dp, d, d, _dp, i],
        "tdks_batch_steps": [v, i, _dp],
        "tdks_batch_stats": [v, C.POINTER(i64), C.POINTER(i), i],
        "tdks_batch_last_error": [v],
        "tdks_batch_set_timing": [v, i],
        "tdks_batch_phase_ms": [v, _dp, C.POINTER(i)],
        "tdks_batch_profile_pass": [v, _dp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = (C.c_char_p if name in ("tdks_last_error", "tdks_status_string",
                                             "tdks_batch_last_error")
                     else C.c_void_p if name == "tdks_batch_stream" else C.c_int)
    _lib = L
    return L


def exported_symbols() -> list:
    return [n for n in ("tdks_create", "tdks_destroy", "tdks_set_stream", "tdks_sizes",
                        "tdks_set_cg", "tdks_set_potential", "tdks_nuclear_potential",
                        "tdks_apply_H", "tdks_density", "tdks_dipole", "tdks_hartree", "tdks_xc",
                        "tdks_expm", "tdks_kick", "tdks_init_propagation", "tdks_magnus_step",
                        "tdks_propagate_host", "tdks_set_timing", "tdks_get_counters",
                        "tdks_fma_probe", "tdks_contraction_probe",
                        "tdks_dipole_noalloc", "tdks_objective_forward",
                        "tdks_objective_backward", "tdks_set_kb", "tdks_kb_info", "tdks_set_lanczos",
                        "tdks_set_apply_tile", "tdks_set_f32_stages", "tdks_set_mixed", "tdks_set_device_loop",
                        "tdks_magnus_step_sc", "tdks_spectrum", "tdks_apply_H_gll",
                        "tdks_nuclear_potential_nodes",
                        "tdks_batch_create", "tdks_batch_destroy",
                        "tdks_batch_stream", "tdks_batch_sizes", "tdks_batch_set_orbitals",
                        "tdks_batch_get_orbitals", "tdks_batch_kick", "tdks_batch_init",
                        "tdks_batch_tune", "tdks_batch_tune_kmax", "tdks_batch_set_kb", "tdks_batch_steps",
                        "tdks_batch_stats",
                        "tdks_batch_last_error", "tdks_batch_set_timing", "tdks_batch_phase_ms",
                        "tdks_batch_profile_pass",
                        "tdks_last_error", "tdks_status_string")]


def _darr(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _dev(t: torch.Tensor, dtype, what: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TDKSError(f"{what}: expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TDKSError(f"{what}: expected a contiguous {dtype} tensor")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def dipole_noalloc(rho: torch.Tensor, X, Y, Z, p: int) -> np.ndarray:
    """tdks_dipole_noalloc: the dipole without a context and without any device
    allocation (fixed scratch inside the library); calls must not overlap.

    The C entry point reads nx*ny*nz*(p+1)^3 doubles from rho and has no length
    argument, so the length is checked here before anything reaches the library.
    The call runs on rho's device and on that device's current stream."""
    Xa, Ya, Za = _darr(X), _darr(Y), _darr(Z)
    n_e = (len(Xa) - 1) * (len(Ya) - 1) * (len(Za) - 1)
    if not isinstance(rho, torch.Tensor) or n_e < 1 or rho.numel() != n_e * (int(p) + 1) ** 3:
        raise TDKSError(f"tdks_dipole_noalloc: rho must hold nx*ny*nz*(p+1)^3 = "
                        f"{max(n_e, 0) * (int(p) + 1) ** 3} values")
    ptr = _dev(rho, torch.float64, "rho")
    d = np.zeros(3)
    with torch.cuda.device(rho.device):
        st = lib().tdks_dipole_noalloc(ptr, len(Xa) - 1, len(Ya) - 1, len(Za) - 1, _ptr(Xa),
                                       _ptr(Ya), _ptr(Za), int(p),
                                       C.c_void_p(torch.cuda.current_stream(rho.device).cuda_stream),
                                       _ptr(d))
    if st != 0:
        raise TDKSError(f"tdks_dipole_noalloc: {lib().tdks_status_string(st).decode()}")
    return d


def fma_probe(prec: int, ctas_per_sm: int = 8, iters: int = 16384, reps: int = 10):
    """tdks_fma_probe on the current device and stream: (TFLOP/s, ms per launch)."""
    tf, ms = np.zeros(1), np.zeros(1)
    st = lib().tdks_fma_probe(int(prec), int(ctas_per_sm), int(iters), int(reps),
                              C.c_void_p(_stream()), _ptr(tf), _ptr(ms))
    if st != 0:
        raise TDKSError(f"tdks_fma_probe: {lib().tdks_status_string(st).decode()}")
    return float(tf[0]), float(ms[0])


def contraction_probe(variant: int, op, x: torch.Tensor, reps: int, out: Optional[torch.Tensor] = None):
    """tdks_contraction_probe on x's device and current stream: (M^reps x, ms per launch).
    variant 0 FP32, 1 double-float, 2 BF16 tensor cores, 3 three-TF32 tensor cores."""
    opa = _darr(op)
    P1 = opa.shape[0]
    if x.dim() != 2 or x.shape[1] != P1 or x.shape[0] % 512:
        raise TDKSError("tdks_contraction_probe: x must be [n_lines][P1] with n_lines a multiple of 512")
    out = torch.empty_like(x) if out is None else out
    ms = np.zeros(1)
    with torch.cuda.device(x.device):
        st = lib().tdks_contraction_probe(int(variant), int(P1), _ptr(opa), _dev(x, torch.float64, "x"),
                                          _dev(out, torch.float64, "out"), int(x.shape[0]), int(reps),
                                          C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream),
                                          _ptr(ms))
    if st != 0:
        raise TDKSError(f"tdks_contraction_probe: {lib().tdks_status_string(st).decode()}")
    return out, float(ms[0])


class Context:
    """Owns a tdks_ctx.  Mirrors tdks_create / tdks_destroy; methods mirror the
    remaining entry points (tdks_<name>)."""

    def __init__(self, X, Y, Z, p: int, n_orb: int, occ, atom_R=None, atom_Z=None,
                 nuc_kind: str = "none", nuc_param: float = 0.0, hartree: bool = True,
                 xc: bool = True, nq: int = 0):
        L = lib()
        self._keep = [_darr(X), _darr(Y), _darr(Z), _darr(occ)]
        R = _darr(atom_R if atom_R is not None else np.zeros((0, 3))).reshape(-1)
        Zc = _darr(atom_Z if atom_Z is not None else np.zeros(0))
        self._keep += [R, Zc]
        m = MeshDesc(len(X) - 1, len(Y) - 1, len(Z) - 1, _ptr(self._keep[0]), _ptr(self._keep[1]),
                     _ptr(self._keep[2]), int(p), int(nq))
        s = SystemDesc(int(n_orb), _ptr(self._keep[3]), len(Zc), _ptr(R) if len(Zc) else None,
                       _ptr(Zc) if len(Zc) else None, NUC_KIND[nuc_kind], float(nuc_param),
                       int(bool(hartree)), int(bool(xc)))
        h = C.c_void_p()
        st = L.tdks_create(C.byref(m), C.byref(s), C.c_void_p(_stream()), C.byref(h))
        if st != 0:
            raise TDKSError(f"tdks_create: {L.tdks_status_string(st).decode()}")
        self.h = h
        self.n_orb = int(n_orb)
        ni, ne, nq3 = C.c_int64(), C.c_int64(), C.c_int()
        L.tdks_sizes(h, C.byref(ni), C.byref(ne), C.byref(nq3))
        self.n_int, self.n_elem, self.nq3 = ni.value, ne.value, nq3.value

    @classmethod
    def from_config(cls, cfg):
        return cls(cfg.X, cfg.Y, cfg.Z, cfg.p, cfg.n_orb, cfg.occ, cfg.atom_R, cfg.atom_Z,
                   cfg.nuc_kind, cfg.nuc_param, cfg.hartree, cfg.xc, cfg.nq)

    def _check(self, st: int, name: str):
        if st != 0:
            L = lib()
            raise TDKSError(f"{name}: {L.tdks_status_string(st).decode()}: "
                            f"{L.tdks_last_error(self.h).decode()}")

    def _sync_stream(self):
        lib().tdks_set_stream(self.h, C.c_void_p(_stream()))

    def close(self):
        if getattr(self, "h", None):
            lib().tdks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, on: bool):
        self._check(lib().tdks_set_timing(self.h, int(bool(on))), "tdks_set_timing")

    def set_lanczos(self, reorth: bool):
        self._check(lib().tdks_set_lanczos(self.h, int(bool(reorth))), "tdks_set_lanczos")

    def set_device_loop(self, on: bool):
        """tdks_set_device_loop: Lanczos iterations of a sub-step as one graph launch."""
        self._check(lib().tdks_set_device_loop(self.h, int(bool(on))), "tdks_set_device_loop")

    def set_mixed(self, relax: float):
        """tdks_set_mixed: FP32 products once every Lanczos estimate <= relax * tol."""
        self._check(lib().tdks_set_mixed(self.h, float(relax)), "tdks_set_mixed")

    def set_apply_tile(self, orbs_per_cta: int):
        """tdks_set_apply_tile: orbitals per CTA of the element kernel (0: automatic)."""
        self._check(lib().tdks_set_apply_tile(self.h, int(orbs_per_cta)), "tdks_set_apply_tile")

    def set_f32_stages(self, mask: int):
        """tdks_set_f32_stages: stages of the double-float apply run in FP32 (study; 0: none)."""
        self._check(lib().tdks_set_f32_stages(self.h, int(mask)), "tdks_set_f32_stages")

    def get_counters(self, reset: bool = False) -> dict:
        c = Counters()
        self._check(lib().tdks_get_counters(self.h, C.byref(c), int(bool(reset))),
                    "tdks_get_counters")
        return {k: getattr(c, k) for k, _ in Counters._fields_}

    # -- allocation helpers (torch owns the memory) -------------------------
    def empty_orbitals(self, n_orb: Optional[int] = None) -> torch.Tensor:
        return torch.empty((n_orb or self.n_orb, self.n_int), dtype=torch.complex128, device="cuda")

    def empty_field(self) -> torch.Tensor:
        return torch.empty((self.n_elem, self.nq3), dtype=torch.float64, device="cuda")

    # -- entry points ---------------------------------------------------------
    def set_cg(self, tol: float, maxit: int = 5000, precond: int = PRECOND_FDM):
        self._check(lib().tdks_set_cg(self.h, tol, maxit, precond), "tdks_set_cg")

    def set_potential(self, v_q: torch.Tensor):
        self._sync_stream()
        self._check(lib().tdks_set_potential(self.h, _dev(v_q, torch.float64, "v_q")),
                    "tdks_set_potential")

    def nuclear_potential(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = self.empty_field() if out is None else out
        self._sync_stream()
        self._check(lib().tdks_nuclear_potential(self.h, _dev(out, torch.float64, "out")),
                    "tdks_nuclear_potential")
        return out

    def apply_H(self, psi: torch.Tensor, out: Optional[torch.Tensor] = None, prec: int = FP64):
        out = torch.empty_like(psi) if out is None else out
        self._sync_stream()
        self._check(lib().tdks_apply_H(self.h, _dev(psi, torch.complex128, "psi"),
                                       _dev(out, torch.complex128, "out"), psi.shape[0], prec),
                    "tdks_apply_H")
        return out

    def density(self, psi: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = self.empty_field() if out is None else out
        self._sync_stream()
        self._check(lib().tdks_density(self.h, _dev(psi, torch.complex128, "psi"), psi.shape[0],
                                       _dev(out, torch.float64, "rho")), "tdks_density")
        return out

    def dipole(self, rho: torch.Tensor) -> np.ndarray:
        d = np.zeros(3)
        self._sync_stream()
        self._check(lib().tdks_dipole(self.h, _dev(rho, torch.float64, "rho"), _ptr(d)),
                    "tdks_dipole")
        return d

    def hartree(self, rho: torch.Tensor, out: Optional[torch.Tensor] = None):
        out = self.empty_field() if out is None else out
        it = C.c_int()
        self._sync_stream()
        self._check(lib().tdks_hartree(self.h, _dev(rho, torch.float64, "rho"),
                                       _dev(out, torch.float64, "vh"), C.byref(it)), "tdks_hartree")
        return out, it.value

    def xc(self, rho: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = self.empty_field() if out is None else out
        self._sync_stream()
        self._check(lib().tdks_xc(self.h, _dev(rho, torch.float64, "rho"),
                                  _dev(out, torch.float64, "vxc")), "tdks_xc")
        return out

    def expm(self, psi: torch.Tensor, tau: float, tol: float = 1e-10, k_max: int = 64,
             prec: int = FP64, out: Optional[torch.Tensor] = None):
        out = torch.empty_like(psi) if out is None else out
        k = (C.c_int * psi.shape[0])()
        self._sync_stream()
        self._check(lib().tdks_expm(self.h, _dev(psi, torch.complex128, "psi"),
                                    _dev(out, torch.complex128, "out"), psi.shape[0], tau, tol,
                                    k_max, prec, k), "tdks_expm")
        return out, list(k)

    def kick(self, psi: torch.Tensor, kappa: float, direction: Sequence[float]):
        d = _darr(direction)
        self._sync_stream()
        self._check(lib().tdks_kick(self.h, _dev(psi, torch.complex128, "psi"), psi.shape[0],
                                    kappa, _ptr(d)), "tdks_kick")
        return psi

    def init_propagation(self, psi: torch.Tensor) -> np.ndarray:
        d = np.zeros(3)
        self._sync_stream()
        self._check(lib().tdks_init_propagation(self.h, _dev(psi, torch.complex128, "psi"),
                                                psi.shape[0], _ptr(d)), "tdks_init_propagation")
        return d

    def magnus_step(self, psi: torch.Tensor, dt: float, E_quarter=(0, 0, 0), E_half=(0, 0, 0),
                    tol: float = 1e-10, k_max: int = 64, prec: int = FP64) -> dict:
        eq, eh = _darr(E_quarter), _darr(E_half)
        st = Stats()
        self._sync_stream()
        self._check(lib().tdks_magnus_step(self.h, _dev(psi, torch.complex128, "psi"),
                                           psi.shape[0], dt, _ptr(eq), _ptr(eh), tol, k_max, prec,
                                           C.byref(st)), "tdks_magnus_step")
        return st.as_dict()

    def propagate_host(self, psi_in: torch.Tensor, psi_out: torch.Tensor, n_steps: int,
                       dt: float, E: Optional[np.ndarray] = None, init: bool = True,
                       tol: float = 1e-10, k_max: int = 64, prec: int = FP64) -> np.ndarray:
        """Host-buffer path: psi_in/psi_out are CPU complex128 tensors (pinned for speed)."""
        for t, nm in ((psi_in, "psi_in"), (psi_out, "psi_out")):
            if t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous():
                raise TDKSError(f"{nm}: expected a contiguous CPU complex128 tensor")
        Eh = None if E is None else _darr(E).reshape(n_steps, 6)
        dip = np.zeros((max(n_steps, 1), 3))
        self._sync_stream()
        self._check(lib().tdks_propagate_host(
            self.h, psi_in.data_ptr(), psi_out.data_ptr(), psi_in.shape[0], int(init), n_steps, dt,
            None if Eh is None else Eh.ctypes.data, tol, k_max, prec, dip.ctypes.data),
            "tdks_propagate_host")
        return dip[:n_steps]

    def magnus_step_sc(self, psi: torch.Tensor, dt: float, E_half=(0, 0, 0), tol: float = 1e-10,
                       k_max: int = 64, prec: int = FP64, sc_tol: float = 1e-10,
                       sc_maxit: int = 50) -> dict:
        eh = _darr(E_half)
        st = Stats()
        it = C.c_int()
        self._sync_stream()
        self._check(lib().tdks_magnus_step_sc(self.h, _dev(psi, torch.complex128, "psi"), psi.shape[0],
                                              dt, _ptr(eh), tol, k_max, prec, sc_tol, sc_maxit,
                                              C.byref(st), C.byref(it)), "tdks_magnus_step_sc")
        out = st.as_dict()
        out["iterations"] = it.value
        return out

    def nuclear_potential_nodes(self) -> torch.Tensor:
        out = torch.empty(self.n_int, dtype=torch.float64, device="cuda")
        self._sync_stream()
        self._check(lib().tdks_nuclear_potential_nodes(self.h, out.data_ptr()),
                    "tdks_nuclear_potential_nodes")
        return out

    def apply_H_gll(self, psi: torch.Tensor, v_nodes: torch.Tensor,
                    out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = torch.empty_like(psi) if out is None else out
        self._sync_stream()
        self._check(lib().tdks_apply_H_gll(self.h, _dev(psi, torch.complex128, "psi"),
                                           _dev(v_nodes, torch.float64, "v_nodes"),
                                           _dev(out, torch.complex128, "out"), psi.shape[0]),
                    "tdks_apply_H_gll")
        return out

    def set_kb(self, R, a: float = 1.0, b: float = 0.8, c=(-2.0, -1.0), lmax: int = 1):
        """Kleinman-Bylander projectors on the atoms at R ([n_atoms, 3]); R empty removes them."""
        Rh = _darr(R).reshape(-1)
        ch = _darr(c).reshape(2)
        self._sync_stream()
        self._check(lib().tdks_set_kb(self.h, len(Rh) // 3, _ptr(Rh) if len(Rh) else None, a, b,
                                      _ptr(ch), lmax), "tdks_set_kb")

    def kb_info(self) -> dict:
        n = C.c_int()
        self._check(lib().tdks_kb_info(self.h, C.byref(n), None, None, None), "tdks_kb_info")
        h = np.zeros(max(n.value, 1))
        nc, nv = C.c_int64(), C.c_int64()
        self._check(lib().tdks_kb_info(self.h, C.byref(n), _ptr(h), C.byref(nc), C.byref(nv)),
                    "tdks_kb_info")
        return {"n_proj": n.value, "h": h[:n.value], "n_covered": nc.value, "n_values": nv.value}

    def objective_forward(self, psi0: torch.Tensor, E: np.ndarray, w, e, dt: float,
                          ckpt_every: int = 10, tol: float = 1e-10, k_max: int = 64,
                          prec: int = FP64):
        """J = sum_n w_n (e . mu_n)^2 over the propagation from psi0 with field samples
        E ([n_steps, 6]); returns (J, dipoles [n_steps + 1, 3]).  Keeps checkpoints
        for objective_backward."""
        Eh = _darr(E).reshape(-1, 6)
        n = Eh.shape[0]
        wh = _darr(w).reshape(-1)
        if wh.shape[0] != n + 1:
            raise TDKSError("objective_forward: w needs n_steps + 1 weights")
        eh = _darr(e).reshape(3)
        J = C.c_double(0.0)
        dip = np.zeros((n + 1, 3))
        self._sync_stream()
        self._check(lib().tdks_objective_forward(
            self.h, _dev(psi0, torch.complex128, "psi0"), psi0.shape[0], n, dt, _ptr(Eh), _ptr(wh),
            _ptr(eh), ckpt_every, tol, k_max, prec, C.byref(J), _ptr(dip)), "tdks_objective_forward")
        self._n_obj_steps = n
        return J.value, dip

    def objective_backward(self, n_s: int = 8) -> np.ndarray:
        """dJ/dE ([n_steps, 6]) of the last objective_forward call."""
        n = getattr(self, "_n_obj_steps", 0)
        g = np.zeros((max(n, 1), 6))
        self._sync_stream()
        self._check(lib().tdks_objective_backward(self.h, n_s, _ptr(g)), "tdks_objective_backward")
        return g[:n]


class DipoleObjective(torch.autograd.Function):
    """J(E) = sum_n w_n (e . mu_n)^2 as a differentiable function of the field samples
    E ([n_steps, 6], float64, any device): forward propagates on the GPU with
    checkpoints, backward runs the adjoint sweep (no autograd tape of the propagation).

        J = DipoleObjective.apply(E, ctx, psi0, w, e, dt, ckpt_every, tol, k_max, prec, n_s)
    """

    @staticmethod
    def forward(fctx, E, tdctx, psi0, w, e, dt, ckpt_every=10, tol=1e-10, k_max=64, prec=FP64,
                n_s=8):
        J, _ = tdctx.objective_forward(psi0, E.detach().cpu().numpy(), w, e, dt, ckpt_every, tol,
                                       k_max, prec)
        fctx.tdctx = tdctx
        fctx.n_s = n_s
        fctx.E_meta = (E.device, E.dtype, E.shape)
        return torch.tensor(J, dtype=E.dtype, device=E.device)

    @staticmethod
    def backward(fctx, gJ):
        dev, dt_, shape = fctx.E_meta
        g = fctx.tdctx.objective_backward(fctx.n_s)
        gE = torch.from_numpy(g).to(device=dev, dtype=dt_).reshape(shape) * gJ
        return (gE,) + (None,) * 10


def _descs(cfg, keep):
    """tdks_mesh_desc / tdks_system_desc of a workload config (arrays kept alive in keep)."""
    arrs = [_darr(cfg.X), _darr(cfg.Y), _darr(cfg.Z), _darr(cfg.occ)]
    R = _darr(cfg.atom_R if cfg.atom_R is not None else np.zeros((0, 3))).reshape(-1)
    Zc = _darr(cfg.atom_Z if cfg.atom_Z is not None else np.zeros(0))
    keep += arrs + [R, Zc]
    m = MeshDesc(len(cfg.X) - 1, len(cfg.Y) - 1, len(cfg.Z) - 1, _ptr(arrs[0]), _ptr(arrs[1]),
                 _ptr(arrs[2]), int(cfg.p), int(cfg.nq))
    s = SystemDesc(int(cfg.n_orb), _ptr(arrs[3]), len(Zc), _ptr(R) if len(Zc) else None,
                   _ptr(Zc) if len(Zc) else None, NUC_KIND[cfg.nuc_kind], float(cfg.nuc_param),
                   int(bool(cfg.hartree)), int(bool(cfg.xc)))
    return m, s


def spectrum(dip, dt: float, kappa: float, direction, window: float, omega):
    """(alpha(omega) complex array, S(omega)) of a kicked dipole series (tdks_spectrum)."""
    d = _darr(dip).reshape(-1, 3)
    di = _darr(direction).reshape(3)
    om = _darr(omega).reshape(-1)
    a = np.zeros(2 * len(om))
    S = np.zeros(len(om))
    torch.cuda.current_stream().synchronize()
    st = lib().tdks_spectrum(_ptr(d), d.shape[0], dt, kappa, _ptr(di), window, _ptr(om), len(om),
                             _ptr(a), _ptr(S))
    if st != 0:
        raise TDKSError(f"tdks_spectrum: {lib().tdks_status_string(st).decode()}")
    return a[0::2] + 1j * a[1::2], S


class Batch:
    """Owns a tdks_batch: many independent systems advanced together, one CUDA graph
    per step (tdks_batch_* entry points).  All work runs on the batch's own stream."""

    def __init__(self, cfgs, dts, prec: int = FP64, tol: float = 1e-10, k_max: int = 64):
        L = lib()
        keep = []
        ms, ss = [], []
        for cfg in cfgs:
            m, s = _descs(cfg, keep)
            ms.append(m)
            ss.append(s)
        n = len(cfgs)
        M = (MeshDesc * n)(*ms)
        S = (SystemDesc * n)(*ss)
        dt = _darr(dts)
        h = C.c_void_p()
        torch.cuda.current_stream().synchronize()
        st = L.tdks_batch_create(n, C.cast(M, C.c_void_p), C.cast(S, C.c_void_p), _ptr(dt), prec,
                                 tol, k_max, C.byref(h))
        if st != 0:
            raise TDKSError(f"tdks_batch_create: {L.tdks_status_string(st).decode()}: "
                            f"{L.tdks_batch_last_error(None).decode()}")
        self.h = h
        self.n_sys = n
        self.prec = prec
        self.sizes = []
        for k in range(n):
            ni, ne, nq3, no = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
            L.tdks_batch_sizes(h, k, C.byref(ni), C.byref(ne), C.byref(nq3), C.byref(no))
            self.sizes.append({"n_int": ni.value, "n_elem": ne.value, "nq3": nq3.value,
                               "n_orb": no.value})

    def _check(self, st: int, name: str):
        if st != 0:
            L = lib()
            raise TDKSError(f"{name}: {L.tdks_status_string(st).decode()}: "
                            f"{L.tdks_batch_last_error(self.h).decode()}")

    @property
    def stream(self) -> int:
        return int(lib().tdks_batch_stream(self.h) or 0)

    def close(self):
        if getattr(self, "h", None):
            lib().tdks_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_orbitals(self, k: int, psi: torch.Tensor):
        z = self.sizes[k]
        if tuple(psi.shape) != (z["n_orb"], z["n_int"]):
            raise TDKSError(f"set_orbitals: expected shape {(z['n_orb'], z['n_int'])}")
        torch.cuda.current_stream().synchronize()
        self._check(lib().tdks_batch_set_orbitals(self.h, k, _dev(psi, torch.complex128, "psi")),
                    "tdks_batch_set_orbitals")

    def get_orbitals(self, k: int) -> torch.Tensor:
        z = self.sizes[k]
        out = torch.empty((z["n_orb"], z["n_int"]), dtype=torch.complex128, device="cuda")
        torch.cuda.current_stream().synchronize()
        self._check(lib().tdks_batch_get_orbitals(self.h, k, out.data_ptr()), "tdks_batch_get_orbitals")
        return out

    def kick(self, kappa, directions):
        ka = _darr(kappa).reshape(self.n_sys)
        di = _darr(directions).reshape(self.n_sys, 3)
        self._check(lib().tdks_batch_kick(self.h, _ptr(ka), _ptr(di)), "tdks_batch_kick")

    def init(self) -> np.ndarray:
        d = np.zeros((self.n_sys, 3))
        self._check(lib().tdks_batch_init(self.h, _ptr(d)), "tdks_batch_init")
        return d

    def tune(self, reps: int = 3) -> list:
        cap = 64
        out = (TileChoice * cap)()
        n = C.c_int()
        self._check(lib().tdks_batch_tune(self.h, reps, C.cast(out, C.c_void_p), cap, C.byref(n)),
                    "tdks_batch_tune")
        return [{"p": t.p, "n_orb": t.n_orb, "elems_per_cta": t.elems_per_cta,
                 "orbs_per_item": t.orbs_per_item, "ms": t.ms} for t in out[:n.value]]

    def set_kb(self, k: int, R, a: float = 1.0, b: float = 0.8, c=(-2.0, -1.0), lmax: int = 1):
        """Kleinman-Bylander projectors on the atoms at R ([n_atoms, 3]) for system k of
        the batch (as Context.set_kb); R empty removes them."""
        Rh = _darr(R).reshape(-1)
        ch = _darr(c).reshape(2)
        self._check(lib().tdks_batch_set_kb(self.h, k, len(Rh) // 3, _ptr(Rh) if len(Rh) else None, a, b,
                                            _ptr(ch), lmax), "tdks_batch_set_kb")

    def tune_kmax(self, k_cap: int = 128, mem_budget: int = -1) -> list:
        """Per-system Krylov caps after a step: k_cap for the systems whose last
        exponential took sub-steps, within mem_budget bytes of added basis (< 0:
        half of the free device memory); returns the caps [n_sys]."""
        out = (C.c_int * self.n_sys)()
        self._check(lib().tdks_batch_tune_kmax(self.h, k_cap, mem_budget, out), "tdks_batch_tune_kmax")
        return list(out)

    def steps(self, n_steps: int) -> np.ndarray:
        """n_steps steps of every system; dipoles [n_steps, n_sys, 3]."""
        d = np.zeros((max(n_steps, 1), self.n_sys, 3))
        self._check(lib().tdks_batch_steps(self.h, n_steps, _ptr(d)), "tdks_batch_steps")
        return d[:n_steps]

    def set_timing(self, on: bool):
        self._check(lib().tdks_batch_set_timing(self.h, int(bool(on))), "tdks_batch_set_timing")

    def phase_ms(self) -> dict:
        """Device time of the last step's phases and the loop passes of its exponentials."""
        ms = np.zeros(5)
        passes = (C.c_int * 2)()
        self._check(lib().tdks_batch_phase_ms(self.h, _ptr(ms), passes), "tdks_batch_phase_ms")
        names = ("predictor", "half_exp", "corrector_fields", "full_exp", "history_dipole")
        return {**dict(zip(names, ms.tolist())), "passes": list(passes)}

    def profile_pass(self) -> dict:
        """Kernel-group device times of the half-step exponential, re-run outside the graph."""
        ms = np.zeros(6)
        self._check(lib().tdks_batch_profile_pass(self.h, _ptr(ms)), "tdks_batch_profile_pass")
        return dict(zip(("norms", "apply", "alpha", "assembly", "small_exp", "recombination"),
                        ms.tolist()))

    def stats(self, reset: bool = False) -> dict:
        dof, k = C.c_int64(), C.c_int()
        self._check(lib().tdks_batch_stats(self.h, C.byref(dof), C.byref(k), int(reset)),
                    "tdks_batch_stats")
        return {"dof_applies": dof.value, "k_max_seen": k.value}
