"""Python binding of the C ABI in include/pstd.h (argument marshalling only).

Every computation runs in libpstd.so on the GPU; this module converts arguments
(numpy arrays for host memory, torch CUDA tensors for device memory), calls the
C entry points of the same names and turns status codes into exceptions.  There is
no CPU fallback: if the library is missing or fails to load, the import raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, byref, c_double, c_int, c_long, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpstd.so")

F32, F64 = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
DTYPE_F32, DTYPE_F64 = 0, 1
ABC_POLY, ABC_POSCHL_TELLER = 0, 1
XY_SEPARATE, XY_PLANE, XY_CLUSTER = 0, 1, 2
LINE_PLAIN, LINE_PIPELINED, LINE_TMA = 0, 1, 2
TFSF_EXACT, TFSF_PAPER = 0, 1
ENV_CW_RAMP = 0
FIELD_CURRENT, FIELD_PREVIOUS, FIELD_SCATTERED = 0, 1, 2
MAX_FREQ = 16

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSTABLE", 5: "ESTATE", 6: "ENONFINITE", 7: "ETIMEOUT"}
KERNELS = {"xpass": 0, "ypass": 1, "zpass": 2, "xypass": 3, "prepare": 4, "transform": 5, "far_field": 6, "source": 7,
           "aux": 8}


class PstdError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.code = STATUS.get(status, str(status))
        super().__init__(f"{where}: PSTD_{self.code}: {message}")


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("n", c_int * 3), ("d", c_double * 3), ("dt", c_double), ("hbar", c_double), ("mass", c_double),
        ("precision", c_int), ("batch", c_int), ("abc_cells", c_int * 3), ("abc_profile", c_int),
        ("abc_param", c_double * 2), ("tfsf_lo", c_int * 3), ("tfsf_hi", c_int * 3), ("taper_cells", c_int),
        ("tfsf_mode", c_int), ("huygens_lo", c_int * 3), ("huygens_hi", c_int * 3), ("stream", c_void_p),
    ]


_SIGS = {
    "pstd_create_grid": (c_int, [POINTER(GridDesc), POINTER(c_void_p)]),
    "pstd_destroy_grid": (c_int, [c_void_p]),
    "pstd_set_potential": (c_int, [c_void_p, c_void_p, c_int, c_int]),
    "pstd_set_incidence": (c_int, [c_void_p, c_int, POINTER(c_double), c_double, c_int, c_double]),
    "pstd_reset": (c_int, [c_void_p]),
    "pstd_huygens_dft": (c_int, [c_void_p, c_int, POINTER(c_double), c_int, c_long, c_long]),
    "pstd_step": (c_int, [c_void_p, c_long]),
    "pstd_transform_to_points": (c_int, [c_void_p, c_int, c_int, c_void_p, c_long, c_void_p, c_int]),
    "pstd_cross_section": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_long, c_void_p, c_void_p, c_int]),
    "pstd_transform_members": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int), c_void_p, c_long, c_void_p, c_int]),
    "pstd_set_transform_order": (c_int, [c_void_p, c_int]),
    "pstd_cross_section_noalloc": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_long, c_void_p, c_void_p]),
    "pstd_get_field": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int]),
    "pstd_set_field": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_long, c_int]),
    "pstd_get_phasors": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int]),
    "pstd_synchronize": (c_int, [c_void_p]),
    "pstd_get_step": (c_int, [c_void_p, POINTER(c_long)]),
    "pstd_get_device": (c_int, [c_void_p, POINTER(c_int)]),
    "pstd_measure_fma_peak": (c_int, [c_int, POINTER(c_double)]),
    "pstd_selftest_bounded_wait": (c_int, [c_double, POINTER(c_double)]),
    "pstd_stability_dt_max": (c_int, [POINTER(GridDesc), c_double, POINTER(c_double)]),
    "pstd_set_timing": (c_int, [c_void_p, c_int]),
    "pstd_kernel_stats": (c_int, [c_void_p, c_int, POINTER(c_long), POINTER(c_double)]),
    "pstd_launch_count": (c_int, [c_void_p, POINTER(c_long)]),
    "pstd_last_error": (ctypes.c_char_p, [c_void_p]),
    "pstd_transform_adjoint": (c_int, [c_void_p, c_int, c_int, c_void_p, c_long, c_void_p, c_void_p, c_int]),
    "pstd_adjoint_gradient": (c_int, [c_void_p, c_long, c_void_p, POINTER(c_int), POINTER(c_int), c_long, c_void_p, c_int]),
    "pstd_set_checkpointing": (c_int, [c_void_p, c_long, c_long]),
    "pstd_set_incidence_packet": (c_int, [c_void_p, c_int, POINTER(c_double), c_double, c_double, c_double]),
    "pstd_set_graphs": (c_int, [c_void_p, c_int]),
    "pstd_set_incidence_aux": (c_int, [c_void_p, c_int, POINTER(c_double), c_double, c_double, c_double, c_long,
                                        c_void_p]),
    "pstd_set_magnetic_field": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int, c_int]),
    "pstd_set_incidence_spinor": (c_int, [c_void_p, c_int, POINTER(c_double), c_double, c_double, POINTER(c_double)]),
    "pstd_graph_replays": (c_int, [c_void_p, POINTER(c_long)]),
    "pstd_set_variants": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
    "pstd_autotune": (c_int, [c_void_p, c_long, POINTER(c_int)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpstd.so (raises if it is missing: there is no fallback).  The in-tree library
    is loaded once and cached; another path is loaded as asked."""
    global _lib
    if path == LIB_PATH and _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def _check(status: int, where: str, handle=None):
    if status != 0:
        msg = load_library().pstd_last_error(handle)
        raise PstdError(status, where, msg.decode() if msg else "")


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


def _ptr(x, dtype=None):
    """(pointer, mem, keep-alive) for a numpy array (host) or a torch CUDA tensor (device)."""
    if _is_cuda_tensor(x):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return c_void_p(x.data_ptr()), MEM_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(c_void_p), MEM_HOST, a


def make_desc(spec, precision: int = F32, batch: int = 1, stream=None) -> GridDesc:
    """Fill a pstd_grid_desc from a GridSpec-like object (see paper_2403_04053_gb300.inputs)."""
    d = GridDesc()
    d.n[:] = list(spec.n)
    d.d[:] = list(spec.d)
    d.dt, d.hbar, d.mass = spec.dt, spec.hbar, spec.mass
    d.precision = precision
    d.batch = batch
    d.abc_cells[:] = list(spec.abc_cells)
    d.abc_profile = ABC_POLY if spec.abc_profile == "poly" else ABC_POSCHL_TELLER
    d.abc_param[:] = list(spec.abc_param)
    d.tfsf_lo[:] = list(spec.tfsf_lo)
    d.tfsf_hi[:] = list(spec.tfsf_hi)
    d.taper_cells = spec.taper_cells
    d.tfsf_mode = TFSF_EXACT if spec.tfsf_mode == "exact" else TFSF_PAPER
    d.huygens_lo[:] = list(spec.huygens_lo)
    d.huygens_hi[:] = list(spec.huygens_hi)
    d.stream = stream
    return d


def measure_fma_peak(precision: int) -> float:
    """Measured FMA peak of the current device in TFLOP/s (pstd_measure_fma_peak)."""
    out = c_double()
    _check(load_library().pstd_measure_fma_peak(int(precision), byref(out)), "pstd_measure_fma_peak")
    return out.value


def selftest_bounded_wait(limit_s: float):
    """(status name, seconds waited) of pstd_selftest_bounded_wait: "ETIMEOUT" when the bounded
    wait on a barrier that nothing arrives on gave up, as it must."""
    out = c_double()
    st = load_library().pstd_selftest_bounded_wait(float(limit_s), byref(out))
    return STATUS.get(st, str(st)), out.value


def stability_dt_max(spec, vmax: float) -> float:
    out = c_double()
    _check(load_library().pstd_stability_dt_max(byref(make_desc(spec)), vmax, byref(out)), "pstd_stability_dt_max")
    return out.value


class Grid:
    """One pstd_grid: the state of `batch` incident waves on one internal model."""

    def __init__(self, spec, precision: int = F32, batch: int = 1, stream="default"):
        self.lib = load_library()
        self.spec = spec
        self.precision = precision
        self.batch = batch
        self.shape = tuple(spec.shape)
        self.ncell = int(np.prod(self.shape))
        self.cdtype = np.complex64 if precision == F32 else np.complex128
        self.stream = _default_stream() if stream == "default" else stream
        self.desc = make_desc(spec, precision, batch, self.stream)
        h = c_void_p()
        _check(self.lib.pstd_create_grid(byref(self.desc), byref(h)), "pstd_create_grid", None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.pstd_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _c(self, status, where):
        _check(status, where, self.h)

    # -- set-up ---------------------------------------------------------------------
    def set_potential(self, V):
        if _is_cuda_tensor(V):
            dtype = DTYPE_F64 if str(V.dtype).endswith("float64") else DTYPE_F32
            p, mem, keep = _ptr(V)
        else:
            V = np.ascontiguousarray(V)
            dtype = DTYPE_F32 if V.dtype == np.float32 else DTYPE_F64
            p, mem, keep = _ptr(V, np.float32 if dtype == DTYPE_F32 else np.float64)
        self._c(self.lib.pstd_set_potential(self.h, p, mem, dtype), "pstd_set_potential")

    def set_incidence(self, b: int, khat, k: float, ramp_time: float, envelope: int = ENV_CW_RAMP):
        kh = (c_double * 3)(*[float(v) for v in khat])
        self._c(self.lib.pstd_set_incidence(self.h, b, kh, float(k), envelope, float(ramp_time)), "pstd_set_incidence")

    def set_incidence_aux(self, b: int, khat, k: float, d_lo: float, dd: float, psi0):
        """Incidence from the 1-D auxiliary wave (pstd_set_incidence_aux); psi0: n1 complex samples
        of the profile at d_lo + m dd, t = 0."""
        kh = (c_double * 3)(*[float(v) for v in khat])
        p = np.ascontiguousarray(psi0, dtype=np.complex128)
        self._c(self.lib.pstd_set_incidence_aux(self.h, b, kh, float(k), float(d_lo), float(dd), p.size,
                                                p.ctypes.data_as(c_void_p)), "pstd_set_incidence_aux")

    def set_magnetic_field(self, B, gamma: float):
        """Spinor coupling gamma sigma . B (pstd_set_magnetic_field); B = (Bx, By, Bz) host arrays."""
        arrs = [np.ascontiguousarray(b, dtype=np.float64) for b in B]
        self._c(self.lib.pstd_set_magnetic_field(self.h, *[a.ctypes.data_as(c_void_p) for a in arrs], float(gamma),
                                                 MEM_HOST, DTYPE_F64), "pstd_set_magnetic_field")

    def set_incidence_spinor(self, p: int, khat, k: float, ramp_time: float, chi):
        """CW incidence of spinor p with spin state chi = (up, down) (pstd_set_incidence_spinor)."""
        kh = (c_double * 3)(*[float(v) for v in khat])
        c = (c_double * 4)(complex(chi[0]).real, complex(chi[0]).imag, complex(chi[1]).real, complex(chi[1]).imag)
        self._c(self.lib.pstd_set_incidence_spinor(self.h, p, kh, float(k), float(ramp_time), c), "pstd_set_incidence_spinor")

    def set_incidence_packet(self, b: int, khat, k: float, sigma: float, d0: float):
        """Gaussian wave-packet incidence of member b (pstd_set_incidence_packet)."""
        kh = (c_double * 3)(*[float(v) for v in khat])
        self._c(self.lib.pstd_set_incidence_packet(self.h, b, kh, float(k), float(sigma), float(d0)),
                "pstd_set_incidence_packet")

    def reset(self):
        self._c(self.lib.pstd_reset(self.h), "pstd_reset")

    def huygens_dft(self, b: int, omegas, first_step: int, n_steps: int):
        om = (c_double * max(1, len(omegas)))(*[float(w) for w in omegas])
        self._c(self.lib.pstd_huygens_dft(self.h, b, om, len(omegas), int(first_step), int(n_steps)), "pstd_huygens_dft")

    # -- stepping -------------------------------------------------------------------
    def step(self, nsteps: int = 1):
        self._c(self.lib.pstd_step(self.h, int(nsteps)), "pstd_step")

    def synchronize(self):
        self._c(self.lib.pstd_synchronize(self.h), "pstd_synchronize")

    def get_step(self) -> int:
        n = c_long()
        self._c(self.lib.pstd_get_step(self.h, byref(n)), "pstd_get_step")
        return n.value

    # -- fields ---------------------------------------------------------------------
    def get_field(self, b: int = 0, which: int = FIELD_CURRENT, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.cdtype)
        p, mem, keep = (c_void_p(out.data_ptr()), MEM_DEVICE, out) if _is_cuda_tensor(out) else (out.ctypes.data_as(c_void_p), MEM_HOST, out)
        self._c(self.lib.pstd_get_field(self.h, b, which, p, mem), "pstd_get_field")
        return out

    def set_field(self, b: int, prev, cur, n: int):
        pp, mp, k1 = _ptr(prev, self.cdtype)
        pc, mc, k2 = _ptr(cur, self.cdtype)
        if mp != mc:
            raise ValueError("prev and cur must both be host arrays or both device tensors")
        self._c(self.lib.pstd_set_field(self.h, b, pp, pc, int(n), mp), "pstd_set_field")

    def _plane_shapes(self):
        nx, ny, nz = self.spec.n
        return [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]

    def phasor_count(self) -> int:
        """complex128 entries of one frequency's phasors (six faces, psi then d psi plane)."""
        return sum(2 * s[0] * s[1] for s in self._plane_shapes())

    def split_phasors(self, buf):
        """Flat phasor-layout array -> six (psi, d psi) plane pairs (views)."""
        out, off = [], 0
        for s in self._plane_shapes():
            m = s[0] * s[1]
            out.append((buf[off:off + m].reshape(s), buf[off + m:off + 2 * m].reshape(s)))
            off += 2 * m
        return out

    def join_phasors(self, pairs) -> np.ndarray:
        """Six (psi, d psi) plane pairs -> flat phasor-layout complex128 array."""
        return np.concatenate([np.asarray(a, dtype=np.complex128).ravel() for pair in pairs for a in pair])

    def get_phasors(self, b: int = 0, f: int = 0):
        """Six (psi, d psi / d axis) plane pairs (complex128), face order 2*axis + side."""
        buf = np.empty(self.phasor_count(), dtype=np.complex128)
        self._c(self.lib.pstd_get_phasors(self.h, b, f, buf.ctypes.data_as(c_void_p), MEM_HOST), "pstd_get_phasors")
        return self.split_phasors(buf)

    # -- discrete adjoint -----------------------------------------------------------
    def transform_adjoint(self, b: int, f: int, xyz, dl_dpsi):
        """Gradient with respect to the scaled phasors (pstd_transform_adjoint).  Host inputs
        give six (psi, d psi) plane pairs; CUDA tensors give a flat complex128 tensor."""
        if _is_cuda_tensor(xyz):
            import torch
            g = dl_dpsi.to(torch.complex128).contiguous()
            out = torch.empty(self.phasor_count(), dtype=torch.complex128, device=xyz.device)
            self._c(self.lib.pstd_transform_adjoint(self.h, b, f, c_void_p(xyz.data_ptr()), int(xyz.shape[0]),
                                                    c_void_p(g.data_ptr()), c_void_p(out.data_ptr()), MEM_DEVICE),
                    "pstd_transform_adjoint")
            return out
        pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        g = np.ascontiguousarray(dl_dpsi, dtype=np.complex128)
        out = np.empty(self.phasor_count(), dtype=np.complex128)
        self._c(self.lib.pstd_transform_adjoint(self.h, b, f, pts.ctypes.data_as(c_void_p), len(pts),
                                                g.ctypes.data_as(c_void_p), out.ctypes.data_as(c_void_p), MEM_HOST),
                "pstd_transform_adjoint")
        return self.split_phasors(out)

    def set_variants(self, fused_xy: int, y_pass: int = 0, z_pass: int = 0, plans: int = 0):
        """Force the step-kernel variants (pstd_set_variants): fused_xy is XY_SEPARATE, XY_PLANE
        or XY_CLUSTER; y_pass and z_pass are LINE_PLAIN, LINE_PIPELINED (y only) or LINE_TMA;
        plans has bit a set for the alternative FFT plan along axis a."""
        self._c(self.lib.pstd_set_variants(self.h, int(fused_xy), int(y_pass), int(z_pass), int(plans)),
                "pstd_set_variants")

    def autotune(self, trial_steps: int = 20):
        """Time the available step-kernel variants and keep the fastest (pstd_autotune);
        returns {"fused_xy": XY_*, "y_pass": LINE_*, "z_pass": LINE_*, "plans": bits}."""
        out = (c_int * 4)()
        self._c(self.lib.pstd_autotune(self.h, int(trial_steps), out), "pstd_autotune")
        return {"fused_xy": int(out[0]), "y_pass": int(out[1]), "z_pass": int(out[2]), "plans": int(out[3])}

    def graph_replays(self) -> int:
        n = c_long()
        self._c(self.lib.pstd_graph_replays(self.h, byref(n)), "pstd_graph_replays")
        return n.value

    def set_graphs(self, enable: bool):
        """CUDA-graph replay of repeated step() runs (pstd_set_graphs; on by default)."""
        self._c(self.lib.pstd_set_graphs(self.h, 1 if enable else 0), "pstd_set_graphs")

    def set_checkpointing(self, interval: int, max_steps: int):
        """Record adjoint checkpoints during step() (pstd_set_checkpointing); interval 0 stops."""
        self._c(self.lib.pstd_set_checkpointing(self.h, int(interval), int(max_steps)), "pstd_set_checkpointing")

    def adjoint_gradient(self, nsteps: int, dl_dphasors, box_lo, box_hi, checkpoint_interval: int = 0):
        """dL/dV on the node box [box_lo, box_hi) (x, y, z) as a [z, y, x] array
        (pstd_adjoint_gradient).  dl_dphasors: one block per (member, frequency), members in
        order and each member's frequencies in order, each block six plane pairs or a flat
        array; or one flat CUDA tensor holding every block (then the result is a CUDA tensor).
        On a batch the members share V, so the gradient is the sum of their contributions."""
        lo = (c_int * 3)(*[int(v) for v in box_lo])
        hi = (c_int * 3)(*[int(v) for v in box_hi])
        shape = (int(box_hi[2]) - int(box_lo[2]), int(box_hi[1]) - int(box_lo[1]), int(box_hi[0]) - int(box_lo[0]))
        if _is_cuda_tensor(dl_dphasors):
            import torch
            g = dl_dphasors.to(torch.complex128).contiguous()
            out = torch.empty(shape, dtype=torch.float64, device=g.device)
            self._c(self.lib.pstd_adjoint_gradient(self.h, int(nsteps), c_void_p(g.data_ptr()), lo, hi, int(checkpoint_interval),
                                                   c_void_p(out.data_ptr()), MEM_DEVICE), "pstd_adjoint_gradient")
            return out
        blocks = [self.join_phasors(x) if isinstance(x, (list, tuple)) else np.asarray(x, dtype=np.complex128).ravel()
                  for x in dl_dphasors]
        g = np.ascontiguousarray(np.concatenate(blocks))
        out = np.empty(shape, dtype=np.float64)
        self._c(self.lib.pstd_adjoint_gradient(self.h, int(nsteps), g.ctypes.data_as(c_void_p), lo, hi, int(checkpoint_interval),
                                               out.ctypes.data_as(c_void_p), MEM_HOST), "pstd_adjoint_gradient")
        return out

    # -- transforms -----------------------------------------------------------------
    def transform_to_points(self, b: int, f: int, xyz, out=None):
        if _is_cuda_tensor(xyz):
            import torch
            M = xyz.shape[0]
            if out is None:
                out = torch.empty(M, dtype=torch.complex128, device=xyz.device)
            self._c(self.lib.pstd_transform_to_points(self.h, b, f, c_void_p(xyz.data_ptr()), M, c_void_p(out.data_ptr()), MEM_DEVICE),
                    "pstd_transform_to_points")
            return out
        pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        res = np.empty(len(pts), dtype=np.complex128) if out is None else out
        self._c(self.lib.pstd_transform_to_points(self.h, b, f, pts.ctypes.data_as(c_void_p), len(pts),
                                                  res.ctypes.data_as(c_void_p), MEM_HOST), "pstd_transform_to_points")
        return res

    def set_transform_order(self, G: int):
        """Gauss-Legendre nodes per cell edge of the surface transform (pstd_set_transform_order)."""
        self._c(self.lib.pstd_set_transform_order(self.h, int(G)), "pstd_set_transform_order")

    def transform_members(self, members, freqs, xyz):
        """Psi of several members at the same points (pstd_transform_members): an array (or a
        CUDA tensor, for device points) of shape (len(members), M)."""
        n = len(members)
        mb = (c_int * n)(*[int(b) for b in members])
        fq = (c_int * n)(*[int(f) for f in freqs])
        if _is_cuda_tensor(xyz):
            import torch
            M = xyz.shape[0]
            out = torch.empty((n, M), dtype=torch.complex128, device=xyz.device)
            self._c(self.lib.pstd_transform_members(self.h, n, mb, fq, c_void_p(xyz.data_ptr()), M, c_void_p(out.data_ptr()),
                                                    MEM_DEVICE), "pstd_transform_members")
            return out
        pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        out = np.empty((n, len(pts)), dtype=np.complex128)
        self._c(self.lib.pstd_transform_members(self.h, n, mb, fq, pts.ctypes.data_as(c_void_p), len(pts),
                                                out.ctypes.data_as(c_void_p), MEM_HOST), "pstd_transform_members")
        return out

    def cross_section(self, b: int, f: int, theta, phi):
        """(dsigma/dOmega, f) at the given directions."""
        if _is_cuda_tensor(theta):
            import torch
            M = theta.shape[0]
            ds = torch.empty(M, dtype=torch.float64, device=theta.device)
            fa = torch.empty(M, dtype=torch.complex128, device=theta.device)
            self._c(self.lib.pstd_cross_section(self.h, b, f, c_void_p(theta.data_ptr()), c_void_p(phi.data_ptr()), M,
                                                c_void_p(ds.data_ptr()), c_void_p(fa.data_ptr()), MEM_DEVICE), "pstd_cross_section")
            return ds, fa
        th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
        ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
        ds = np.empty(len(th))
        fa = np.empty(len(th), dtype=np.complex128)
        self._c(self.lib.pstd_cross_section(self.h, b, f, th.ctypes.data_as(c_void_p), ph.ctypes.data_as(c_void_p), len(th),
                                            ds.ctypes.data_as(c_void_p), fa.ctypes.data_as(c_void_p), MEM_HOST), "pstd_cross_section")
        return ds, fa

    def cross_section_noalloc(self, b: int, f: int, theta, phi, out_dsdo, out_f=None):
        """pstd_cross_section_noalloc: device tensors in and out, no device allocation.

        theta, phi and out_dsdo are float64 CUDA tensors and out_f (optional) a complex128 one,
        all contiguous, on the grid's device, with at least M = theta.shape[0] elements."""
        M = int(theta.shape[0]) if hasattr(theta, "shape") and len(theta.shape) else -1
        dev = self._device_index()
        for name, t, dt in (("theta", theta, "float64"), ("phi", phi, "float64"), ("out_dsdo", out_dsdo, "float64"),
                            ("out_f", out_f, "complex128")):
            if t is None and name == "out_f":
                continue
            if not _is_cuda_tensor(t):
                raise ValueError(f"cross_section_noalloc: {name} must be a CUDA tensor")
            if t.device.index != dev:
                raise ValueError(f"cross_section_noalloc: {name} is on cuda:{t.device.index}, the grid on cuda:{dev}")
            if not str(t.dtype).endswith(dt):
                raise ValueError(f"cross_section_noalloc: {name} must be {dt}, not {t.dtype}")
            if not t.is_contiguous():
                raise ValueError(f"cross_section_noalloc: {name} must be contiguous")
            if t.numel() < M:
                raise ValueError(f"cross_section_noalloc: {name} holds {t.numel()} elements, fewer than M = {M}")
        self._c(self.lib.pstd_cross_section_noalloc(self.h, b, f, c_void_p(theta.data_ptr()), c_void_p(phi.data_ptr()),
                                                    M, c_void_p(out_dsdo.data_ptr()),
                                                    c_void_p(out_f.data_ptr()) if out_f is not None else None),
                "pstd_cross_section_noalloc")
        return out_dsdo, out_f

    def _device_index(self) -> int:
        d = c_int()
        self._c(self.lib.pstd_get_device(self.h, byref(d)), "pstd_get_device")
        return d.value

    # -- instrumentation ------------------------------------------------------------
    def set_timing(self, enable: bool):
        self._c(self.lib.pstd_set_timing(self.h, 1 if enable else 0), "pstd_set_timing")

    def kernel_stats(self, name: str):
        n, ms = c_long(), c_double()
        self._c(self.lib.pstd_kernel_stats(self.h, KERNELS[name], byref(n), byref(ms)), "pstd_kernel_stats")
        return n.value, ms.value

    def launch_count(self) -> int:
        n = c_long()
        self._c(self.lib.pstd_launch_count(self.h, byref(n)), "pstd_launch_count")
        return n.value


def setup_workload(grid: Grid, wl, b: int = 0, inc_index: int = 0, nfreq_omegas=None):
    """Potential, incidence and DFT window of a Workload (inputs.Workload) on member b."""
    inc = wl.incidences[inc_index]
    grid.set_potential(wl.V)
    grid.set_incidence(b, inc.khat, inc.k, inc.ramp_time)
    w0 = wl.spec.hbar * inc.k ** 2 / (2 * wl.spec.mass)
    grid.huygens_dft(b, nfreq_omegas or [w0], wl.window_first, wl.window_len)


def fresnel_field(V, grid: Grid, points, nsteps: int, box_lo, box_hi, checkpoint_interval: int = 0):
    """Psi at `points` after an nsteps run from rest, differentiable with respect to V.

    V: real CUDA tensor [z, y, x] on the grid (the whole potential); points: CUDA tensor
    M x 3 (float64).  Every member of the grid needs its incidence and DFT window; the
    result is Psi of member 0 ([M]) on a one-member grid and of every member ([batch, M])
    otherwise, at the first frequency.  Backward is the discrete adjoint
    (pstd_transform_adjoint of each member, pstd_adjoint_gradient); the gradient is computed
    on the node box [box_lo, box_hi) and is zero outside it."""
    return _FresnelField.apply(V, grid, points, int(nsteps), tuple(box_lo), tuple(box_hi), int(checkpoint_interval))


def _make_fresnel_function():
    import torch

    class FresnelField(torch.autograd.Function):
        @staticmethod
        def forward(ctx, V, grid, points, nsteps, box_lo, box_hi, checkpoint_interval):
            grid.set_potential(V.detach().contiguous())
            # record the checkpoints the backward sweep needs during this run
            K = checkpoint_interval if checkpoint_interval > 0 else int(math.ceil(math.sqrt(nsteps)))
            grid.set_checkpointing(K, nsteps)
            grid.reset()
            grid.step(nsteps)
            if grid.batch == 1:
                psi = grid.transform_to_points(0, 0, points)
            else:
                psi = torch.stack([grid.transform_to_points(b, 0, points) for b in range(grid.batch)])
            ctx.grid, ctx.points, ctx.nsteps = grid, points, nsteps
            ctx.box = (box_lo, box_hi, checkpoint_interval)
            ctx.vshape, ctx.vdtype = V.shape, V.dtype
            return psi

        @staticmethod
        def backward(ctx, grad_psi):
            grid = ctx.grid
            lo, hi, K = ctx.box
            if grid.batch == 1:
                g_ph = grid.transform_adjoint(0, 0, ctx.points, grad_psi)
            else:
                g_ph = torch.cat([grid.transform_adjoint(b, 0, ctx.points, grad_psi[b].contiguous())
                                  for b in range(grid.batch)])
            gbox = grid.adjoint_gradient(ctx.nsteps, g_ph, lo, hi, K)
            gV = torch.zeros(ctx.vshape, dtype=ctx.vdtype, device=gbox.device)
            gV[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = gbox.to(ctx.vdtype)
            return gV, None, None, None, None, None, None

    return FresnelField


class _LazyFunction:
    """Defers `import torch` until the autograd function is first used."""
    _fn = None

    def apply(self, *args):
        if _LazyFunction._fn is None:
            _LazyFunction._fn = _make_fresnel_function()
        return _LazyFunction._fn.apply(*args)


_FresnelField = _LazyFunction()
