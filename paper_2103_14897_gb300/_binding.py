"""ctypes binding of ``liblsplit.so`` (argument marshalling only).

Every step of the computation runs in the library's CUDA kernels; this module
converts problem descriptions and torch device tensors to the plain pointers
and sizes of the C ABI declared in ``include/lsplit.h``.  There is no CPU or
PyTorch fallback: if the shared library is missing or fails to load, every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblsplit.so")

LS_OK, LS_ERR_INVALID, LS_ERR_NOMEM, LS_ERR_CUDA, LS_ERR_TIMEOUT, LS_ERR_STATE = 0, -1, -2, -3, -4, -5
LS_C64, LS_C128 = 0, 1
MASK_MODES = {"init_only": 0, "project": 1}
SCHEMES = {"lie": 0, "strang": 1, "strang_kp": 2, "lie_stoch": 3, "strang_stoch": 4, "yoshida4": 5, "cn_strang": 6,
           "semi_implicit": 7, "random_batch": 8}

# Every entry point declared in include/lsplit.h.
EXPORTS = ["ls_last_error", "ls_create", "ls_destroy", "ls_layout", "ls_index_set",
           "ls_init_gaussian", "ls_step", "ls_step_host", "ls_observables", "ls_density", "ls_samples",
           "ls_adjoint", "ls_mass_noalloc", "ls_batch_create", "ls_batch_destroy", "ls_batch_layout",
           "ls_batch_init_gaussian", "ls_batch_step", "ls_batch_step_host", "ls_batch_observables",
           "ls_batch_config", "ls_batch_debug"]


class LsProblem(C.Structure):
    _fields_ = [
        ("d", C.c_int32),
        ("B1", C.c_double * 4),
        ("B2", C.c_double * 4),
        ("lo1", C.c_int32 * 2), ("q1", C.c_int32 * 2),
        ("lo2", C.c_int32 * 2), ("q2", C.c_int32 * 2),
        ("ecut", C.c_double),
        ("nv1", C.c_int32), ("v1_h", C.POINTER(C.c_int32)), ("v1_c", C.POINTER(C.c_double)),
        ("nv2", C.c_int32), ("v2_h", C.POINTER(C.c_int32)), ("v2_c", C.POINTER(C.c_double)),
        ("dtype", C.c_int32),
        ("frac_den", C.c_int32),
        ("mask_mode", C.c_int32),
        ("shared", C.c_int32),
    ]


class LsObs(C.Structure):
    _fields_ = [("norm", C.c_double), ("ekin", C.c_double), ("epot1", C.c_double),
                ("epot2", C.c_double), ("energy", C.c_double), ("kmean", C.c_double * 2),
                ("overlap_re", C.c_double), ("overlap_im", C.c_double)]


class LsplitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lsplit error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the shared library once; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA extension not built: {path} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = C.CDLL(path)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    lib.ls_last_error.restype = C.c_char_p
    lib.ls_last_error.argtypes = []
    lib.ls_create.argtypes = [C.POINTER(LsProblem), C.POINTER(vp)]
    lib.ls_destroy.argtypes = [vp]
    lib.ls_layout.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.ls_index_set.argtypes = [vp, C.POINTER(C.c_uint8), C.POINTER(i64)]
    lib.ls_density.argtypes = [vp, vp, C.POINTER(C.c_double), i64, C.POINTER(C.c_double), vp]
    lib.ls_init_gaussian.argtypes = [vp, vp, C.POINTER(dbl), dbl, C.POINTER(dbl), vp]
    lib.ls_step.argtypes = [vp, vp, i64, dbl, i32, u64, u64, vp]
    lib.ls_step_host.argtypes = [vp, vp, vp, i64, dbl, i32, u64, u64, vp]
    lib.ls_batch_step_host.argtypes = [vp, vp, vp, i64, dbl, i32, u64, u64, vp]
    lib.ls_observables.argtypes = [vp, vp, vp, C.POINTER(LsObs), vp]
    lib.ls_samples.argtypes = [vp, i32, u64, u64, i32, C.POINTER(i32), C.POINTER(i32), vp]
    lib.ls_adjoint.argtypes = [vp, vp, vp, i64, dbl, i32, u64, u64, C.POINTER(dbl), C.POINTER(dbl),
                               C.POINTER(dbl), C.POINTER(dbl), vp]
    lib.ls_mass_noalloc.argtypes = [vp, i32, i64, i64, i64, vp, vp]
    lib.ls_batch_create.argtypes = [C.POINTER(LsProblem), i32, C.POINTER(vp)]
    lib.ls_batch_destroy.argtypes = [vp]
    lib.ls_batch_layout.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    lib.ls_batch_init_gaussian.argtypes = [vp, vp, C.POINTER(dbl), dbl, C.POINTER(dbl), vp]
    lib.ls_batch_step.argtypes = [vp, vp, i64, dbl, i32, u64, u64, vp]
    lib.ls_batch_observables.argtypes = [vp, vp, C.POINTER(LsObs), vp]
    lib.ls_batch_debug.argtypes = [vp, i32, dbl]
    lib.ls_batch_config.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i32),
                                    C.POINTER(i32), C.POINTER(C.c_float), C.POINTER(i32)]
    for name in EXPORTS[1:]:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != LS_OK:
        raise LsplitError(code, _lib.ls_last_error().decode())


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def make_problem_struct(prob, dtype: str = "c64", frac_den: int = 8, mask_mode: str = "init_only"):
    """Convert a workloads.Problem-like object to the C struct (and keep the
    coefficient arrays alive by returning them too)."""
    s = LsProblem()
    d = int(prob.d)
    s.d = d
    B1 = np.asarray(prob.B1, dtype=np.float64).reshape(d, d)
    B2 = np.asarray(prob.B2, dtype=np.float64).reshape(d, d)
    for i in range(d * d):
        s.B1[i] = float(B1.reshape(-1)[i])
        s.B2[i] = float(B2.reshape(-1)[i])
    for i in range(d):
        s.lo1[i], s.q1[i] = int(prob.lo1[i]), int(prob.q1[i])
        s.lo2[i], s.q2[i] = int(prob.lo2[i]), int(prob.q2[i])
    s.ecut = float(prob.ecut)
    keep = []
    for j, (h, c) in enumerate(((prob.v1_h, prob.v1_c), (prob.v2_h, prob.v2_c))):
        h = np.ascontiguousarray(np.asarray(h, dtype=np.int32).reshape(-1, d))
        cc = np.asarray(c, dtype=np.complex128).reshape(-1)
        cv = np.ascontiguousarray(np.stack([cc.real, cc.imag], axis=1).reshape(-1))
        keep += [h, cv]
        hp = h.ctypes.data_as(C.POINTER(C.c_int32))
        cp = cv.ctypes.data_as(C.POINTER(C.c_double))
        if j == 0:
            s.nv1, s.v1_h, s.v1_c = len(cc), hp, cp
        else:
            s.nv2, s.v2_h, s.v2_c = len(cc), hp, cp
    s.dtype = LS_C64 if dtype == "c64" else LS_C128
    s.frac_den = int(frac_den)
    s.mask_mode = MASK_MODES[mask_mode]
    s.shared = int(getattr(prob, "shared", 0))
    return s, keep


class Context:
    """One lifted problem on the current CUDA device (ls_create / ls_destroy).
    mask_mode: "init_only" (the joint cutoff shapes the initial state only) or
    "project" (every step ends with the projection onto the cutoff)."""

    def __init__(self, prob, dtype: str = "c64", frac_den: int = 8, mask_mode: str = "init_only"):
        lib = load_library()
        self.prob = prob
        self.dtype = dtype
        self.frac_den = frac_den
        st, keep = make_problem_struct(prob, dtype, frac_den, mask_mode)
        h = C.c_void_p()
        _check(lib.ls_create(C.byref(st), C.byref(h)))
        self._h = h
        del keep
        p, r, b = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.ls_layout(self._h, C.byref(p), C.byref(r), C.byref(b)))
        self.pitch, self.rows, self.nbytes = p.value, r.value, b.value
        self.M1, self.M2 = prob.M1, prob.M2

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.ls_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers
    def empty(self, device="cuda"):
        import torch
        dt = torch.complex64 if self.dtype == "c64" else torch.complex128
        return torch.zeros((self.rows, self.pitch), dtype=dt, device=device)

    def from_dense(self, phi: np.ndarray, device="cuda"):
        import torch
        t = self.empty(device)
        dt = np.complex64 if self.dtype == "c64" else np.complex128
        t[:, :self.M1] = torch.from_numpy(np.ascontiguousarray(np.asarray(phi).astype(dt)))
        return t

    def to_dense(self, psi) -> np.ndarray:
        return psi[:, :self.M1].cpu().numpy().astype(np.complex128)

    # -- ABI calls
    def index_set(self):
        mask = np.zeros((self.M2, self.M1), dtype=np.uint8)
        cnt = C.c_int64()
        _check(_lib.ls_index_set(self._h, mask.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(cnt)))
        return mask.astype(bool), cnt.value

    def init_gaussian(self, psi, x0, w, k0, stream=None):
        x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(-1))
        k0 = np.ascontiguousarray(np.asarray(k0, dtype=np.float64).reshape(-1))
        _check(_lib.ls_init_gaussian(self._h, _ptr(psi), x0.ctypes.data_as(C.POINTER(C.c_double)),
                                     float(w), k0.ctypes.data_as(C.POINTER(C.c_double)),
                                     _stream_handle(stream)))

    def step(self, psi, nsteps: int, tau: float, scheme: str = "strang", seed: int = 0,
             step0: int = 0, stream=None):
        _check(_lib.ls_step(self._h, _ptr(psi), int(nsteps), float(tau), SCHEMES[scheme],
                            int(seed) & (2 ** 64 - 1), int(step0), _stream_handle(stream)))

    def step_host(self, host, dev, nsteps: int, tau: float, scheme: str = "strang", seed: int = 0,
                  step0: int = 0, stream=None):
        """ls_step_host: host -> dev, step, dev -> host (host: a CPU tensor of the
        context layout, ideally pinned; dev: a device tensor of the same shape)."""
        if host.is_cuda or host.numel() != dev.numel() or host.dtype != dev.dtype:
            raise ValueError("host must be a CPU tensor matching dev")
        _check(_lib.ls_step_host(self._h, host.data_ptr(), _ptr(dev), int(nsteps), float(tau), SCHEMES[scheme],
                                 int(seed) & (2 ** 64 - 1), int(step0), _stream_handle(stream)))

    def density(self, psi, x, stream=None) -> np.ndarray:
        """psi(x_j) at real-space points x ((npts,) for 1D boxes, (npts, 2)
        for 2D boxes), complex128 array."""
        d = self.prob.d
        xs = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, d))
        out = np.zeros(2 * len(xs), dtype=np.float64)
        _check(_lib.ls_density(self._h, _ptr(psi), xs.ctypes.data_as(C.POINTER(C.c_double)), len(xs),
                               out.ctypes.data_as(C.POINTER(C.c_double)), _stream_handle(stream)))
        return out[0::2] + 1j * out[1::2]

    def observables(self, psi, chi=None, stream=None) -> dict:
        o = LsObs()
        _check(_lib.ls_observables(self._h, _ptr(psi), _ptr(chi), C.byref(o), _stream_handle(stream)))
        return {"norm": o.norm, "ekin": o.ekin, "epot1": o.epot1, "epot2": o.epot2,
                "energy": o.energy, "kmean": [o.kmean[0], o.kmean[1]][: self.prob.d],
                "overlap": complex(o.overlap_re, o.overlap_im)}

    def samples(self, layer: int, seed: int, g0: int, count: int, stream=None) -> np.ndarray:
        S = self.M2 if layer == 1 else self.M1
        p = max(1, S // self.frac_den)
        out = np.zeros((max(count, 1), p), dtype=np.int32)
        pc = C.c_int32()
        _check(_lib.ls_samples(self._h, int(layer), int(seed) & (2 ** 64 - 1), int(g0), int(count),
                               out.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(pc),
                               _stream_handle(stream)))
        assert pc.value == p
        return out[:count]

    def adjoint(self, psi, lam, nsteps: int, tau: float, scheme: str = "strang", seed: int = 0, step0: int = 0,
                stream=None):
        if getattr(self.prob, "shared", 0):
            g1 = np.zeros(self.prob.q1[0] * self.prob.q2[1])
            g2 = np.zeros(self.prob.q2[0] * self.prob.q2[1])
        else:
            g1 = np.zeros(self.M1)
            g2 = np.zeros(self.M2)
        c1 = np.zeros(2 * len(self.prob.v1_c))
        c2 = np.zeros(2 * len(self.prob.v2_c))
        P = C.POINTER(C.c_double)
        _check(_lib.ls_adjoint(self._h, _ptr(psi), _ptr(lam), int(nsteps), float(tau), SCHEMES[scheme],
                               int(seed) & (2 ** 64 - 1), int(step0),
                               g1.ctypes.data_as(P), g2.ctypes.data_as(P),
                               c1.ctypes.data_as(P) if len(c1) else None,
                               c2.ctypes.data_as(P) if len(c2) else None, _stream_handle(stream)))
        return g1, g2, c1.reshape(-1, 2), c2.reshape(-1, 2)


def mass_noalloc(psi, dtype: str, rows: int, cols: int, pitch: int, out, stream=None) -> None:
    """ls_mass_noalloc: sum |psi|^2 into the device double ``out`` without any
    allocation inside the library (fixed device scratch, rows <= 65536)."""
    lib = load_library()
    _check(lib.ls_mass_noalloc(_ptr(psi), LS_C64 if dtype == "c64" else LS_C128, int(rows), int(cols),
                               int(pitch), _ptr(out), _stream_handle(stream)))


class Batch:
    """Independent uneven instances in one device buffer (ls_batch_*)."""

    def __init__(self, probs, dtype: str = "c64"):
        lib = load_library()
        self.probs = list(probs)
        self.dtype = dtype
        arr = (LsProblem * len(self.probs))()
        keep = []
        for i, p in enumerate(self.probs):
            st, k = make_problem_struct(p, dtype)
            arr[i] = st
            keep.append(k)
        h = C.c_void_p()
        _check(lib.ls_batch_create(arr, len(self.probs), C.byref(h)))
        self._h = h
        n = len(self.probs)
        off = (C.c_int64 * (n + 1))()
        pit = (C.c_int64 * n)()
        _check(lib.ls_batch_layout(self._h, off, pit))
        self.offsets = [off[i] for i in range(n + 1)]
        self.pitches = [pit[i] for i in range(n)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.ls_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, device="cuda"):
        import torch
        dt = torch.complex64 if self.dtype == "c64" else torch.complex128
        return torch.zeros(self.offsets[-1], dtype=dt, device=device)

    def view(self, psi, i):
        p = self.probs[i]
        seg = psi[self.offsets[i]:self.offsets[i] + self.pitches[i] * p.M2]
        return seg.view(p.M2, self.pitches[i])[:, :p.M1]

    def set_dense(self, psi, i, phi):
        import torch
        dt = torch.complex64 if self.dtype == "c64" else torch.complex128
        self.view(psi, i).copy_(torch.from_numpy(np.asarray(phi)).to(dt))

    def get_dense(self, psi, i):
        return self.view(psi, i).cpu().numpy().astype(np.complex128)

    def init_gaussian(self, psi, x0, w, k0, stream=None):
        x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(-1))
        k0 = np.ascontiguousarray(np.asarray(k0, dtype=np.float64).reshape(-1))
        _check(_lib.ls_batch_init_gaussian(self._h, _ptr(psi), x0.ctypes.data_as(C.POINTER(C.c_double)),
                                           float(w), k0.ctypes.data_as(C.POINTER(C.c_double)),
                                           _stream_handle(stream)))

    def step(self, psi, nsteps, tau, scheme="strang", seed=0, step0=0, stream=None):
        _check(_lib.ls_batch_step(self._h, _ptr(psi), int(nsteps), float(tau), SCHEMES[scheme],
                                  int(seed) & (2 ** 64 - 1), int(step0), _stream_handle(stream)))

    def step_host(self, host, dev, nsteps, tau, scheme="strang", seed=0, step0=0, stream=None):
        """ls_batch_step_host: host -> dev, nsteps steps, dev -> host."""
        if host.is_cuda or host.numel() != dev.numel() or host.dtype != dev.dtype:
            raise ValueError("host must be a CPU tensor matching dev")
        _check(_lib.ls_batch_step_host(self._h, host.data_ptr(), _ptr(dev), int(nsteps), float(tau),
                                       SCHEMES[scheme], int(seed) & (2 ** 64 - 1), int(step0),
                                       _stream_handle(stream)))

    def observables(self, psi, stream=None):
        out = (LsObs * len(self.probs))()
        _check(_lib.ls_batch_observables(self._h, _ptr(psi), out, _stream_handle(stream)))
        return [{"norm": o.norm, "energy": o.energy} for o in out]

    def config(self) -> dict:
        """ls_batch_config: the compact-kernel launch configuration and the
        autotuner's last timings (ms per two steps per candidate)."""
        t, c, tb, sub, tu, n = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32(16)
        ms = (C.c_float * 16)()
        _check(_lib.ls_batch_config(self._h, C.byref(t), C.byref(c), C.byref(tb), C.byref(sub), C.byref(tu), ms,
                                    C.byref(n)))
        return {"threads": t.value, "ctas_per_sm": c.value, "tile_bytes": tb.value, "tiles_per_item": sub.value,
                "tuned": bool(tu.value), "tune_ms": [ms[k] for k in range(min(n.value, 16))]}

    def debug(self, unmet: bool, timeout_s: float = 1.0):
        _check(_lib.ls_batch_debug(self._h, 1 if unmet else 0, float(timeout_s)))
