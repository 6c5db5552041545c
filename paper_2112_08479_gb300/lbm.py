"""Python binding of the C ABI in include/lbm.h (liblbm.so, built in-tree).

Functions carry the same names as the C entry points and only marshal
arguments; every step of the computation runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: when
liblbm.so is missing or no CUDA device is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field, fields

HERE = os.path.dirname(os.path.abspath(__file__))
RELEASE_LIB_PATH = os.path.join(HERE, "liblbm.so")
DEBUG_LIB_PATH = os.path.join(HERE, "liblbm_debug.so")   # index-checked build (LBM_DEBUG)
# LBM_LIBRARY selects the library: unset or "release", "debug", or a path
_choice = os.environ.get("LBM_LIBRARY", "release")
LIB_PATH = {"release": RELEASE_LIB_PATH, "debug": DEBUG_LIB_PATH}.get(_choice, _choice)

(LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_NOMEM, LBM_ERR_UNSTABLE, LBM_ERR_STATE, LBM_ERR_TIMEOUT,
 LBM_ERR_BOUNDS) = range(8)
LBM_BGK_SMAG_Q19, LBM_CUMULANT_Q27 = 0, 1
LBM_FP32, LBM_FP16S, LBM_BF16S = 0, 1, 2
LBM_FLAG_NO_COLLIDE, LBM_FLAG_PERIODIC_X, LBM_FLAG_PERIODIC_Z, LBM_FLAG_ONE_NODE = 1, 2, 4, 8
LBM_FLAG_TMA_STAGED, LBM_FLAG_TEST_STALL, LBM_FLAG_TEST_BOUNDS = 16, 32, 64
LBM_DEVFLAG_NONFINITE, LBM_DEVFLAG_RHO_NONPOS, LBM_DEVFLAG_TIMEOUT, LBM_DEVFLAG_BOUNDS = 1, 2, 4, 8
# sites of the debug build's index checks (lbm_debug_record)
SITES = {1: "gather", 2: "scatter", 3: "pair load", 4: "pair store", 5: "quad", 6: "staged",
         7: "halo", 8: "adjoint", 9: "state"}

LBM_SCALAR_Q7, LBM_SCALAR_Q6, LBM_SCALAR_Q27 = 0, 1, 2
# 16-bit storage holds the scalar as scale_phi (Phi - LBM_SCALAR_CHI16 w)
LBM_SCALAR_CHI16 = 1.0

MODELS = {"bgk": LBM_BGK_SMAG_Q19, "cumulant": LBM_CUMULANT_Q27}
SCALARS = {"q7": LBM_SCALAR_Q7, "q6": LBM_SCALAR_Q6, "q27": LBM_SCALAR_Q27}
STORAGES = {"fp32": LBM_FP32, "fp16s": LBM_FP16S, "bf16s": LBM_BF16S}


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class lbm_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("model", C.c_int32), ("storage", C.c_int32), ("flags", C.c_int32),
                ("nu", C.c_double), ("D", C.c_double), ("cs_smag", C.c_double),
                ("sc_t", C.c_double), ("gprime", C.c_double), ("eg", C.c_double * 3),
                ("omega_bulk", C.c_double), ("x0", C.c_int32), ("H", C.c_int32),
                ("noise_amp", C.c_double), ("seed", C.c_uint64),
                ("front_threshold", C.c_double), ("scale_f", C.c_double),
                ("scale_phi", C.c_double), ("scalar", C.c_int32), ("x_offset", C.c_int32),
                ("nx_global", C.c_int32), ("pad_", C.c_int32)]


class lbm_diagnostics(C.Structure):
    _fields_ = [("front", C.c_double), ("front_node", C.c_double), ("Fw", C.c_double),
                ("mass_delta", C.c_double), ("scalar_mass", C.c_double),
                ("step", C.c_int64), ("flags", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


# (name, restype, argtypes) of every entry point of include/lbm.h
_P = C.POINTER(lbm_params)
_CTX = C.c_void_p
SIGNATURES = [
    ("lbm_status_string", C.c_char_p, [C.c_int]),
    ("lbm_last_error", C.c_char_p, [_CTX]),
    ("lbm_validate", C.c_int, [_P]),
    ("lbm_workspace_bytes", C.c_size_t, [_P]),
    ("lbm_init", C.c_int, [_P, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("lbm_set_scalar", C.c_int, [_CTX, C.c_void_p]),
    ("lbm_step", C.c_int, [_CTX, C.c_int32]),
    ("lbm_step_save", C.c_int, [_CTX, C.c_void_p]),
    ("lbm_macros", C.c_int, [_CTX, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lbm_diag", C.c_int, [_CTX, C.POINTER(lbm_diagnostics)]),
    ("lbm_fw_accumulate", C.c_int, [_CTX, C.c_void_p, C.c_double]),
    ("lbm_get_state", C.c_int, [_CTX, C.c_void_p]),
    ("lbm_set_state", C.c_int, [_CTX, C.c_void_p, C.c_int64]),
    ("lbm_adjoint_step", C.c_int, [_CTX, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]),
    ("lbm_objective_forward", C.c_int, [_CTX, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    ("lbm_adjoint_segment", C.c_int, [_CTX, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]),
    ("lbm_front_adjoint", C.c_int, [_CTX, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lbm_recompute_segment", C.c_int, [_CTX, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("lbm_adjoint_sweep", C.c_int, [_CTX, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    ("lbm_adjoint_chi0", C.c_int, [_CTX, C.c_void_p, C.c_void_p]),
    ("lbm_diag_static", C.c_int, [_P, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.POINTER(lbm_diagnostics)]),
    ("lbm_halo_bytes", C.c_size_t, [_P]),
    ("lbm_halo_pack", C.c_int, [_CTX, C.c_int32, C.c_void_p]),
    ("lbm_halo_unpack", C.c_int, [_CTX, C.c_int32, C.c_void_p]),
    ("lbm_next_step_odd", C.c_int32, [_CTX]),
    ("lbm_column_max", C.c_int, [_CTX, C.c_void_p]),
    ("lbm_front_of_columns", C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                       C.c_int32, C.c_void_p, C.c_void_p]),
    ("lbm_get_step", C.c_int64, [_CTX]),
    ("lbm_sync", C.c_int, [_CTX]),
    ("lbm_destroy", None, [_CTX]),
    ("lbm_debug_build", C.c_int32, []),
    ("lbm_debug_record", C.c_int, [_CTX, C.POINTER(C.c_int64)]),
]

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Loads liblbm.so; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                              "(the library has no CPU fallback)")
        lib = C.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _check(status: int, ctx=None):
    if status != LBM_OK:
        lib = load()
        msg = lib.lbm_last_error(ctx).decode() if lib else ""
        name = lib.lbm_status_string(status).decode()
        raise LBMError(status, f"{name}: {msg}")


# --- the entry points, same names as the C ABI --------------------------------

def lbm_status_string(s: int) -> str:
    return load().lbm_status_string(s).decode()


def lbm_validate(p: lbm_params) -> int:
    return load().lbm_validate(C.byref(p))


def lbm_workspace_bytes(p: lbm_params) -> int:
    return load().lbm_workspace_bytes(C.byref(p))


def lbm_init(p: lbm_params, workspace_ptr: int, nbytes: int, stream_handle: int):
    ctx = C.c_void_p()
    _check(load().lbm_init(C.byref(p), workspace_ptr, nbytes, stream_handle, C.byref(ctx)))
    return ctx


def lbm_set_scalar(ctx, chi0_ptr: int):
    _check(load().lbm_set_scalar(ctx, chi0_ptr), ctx)


def lbm_step(ctx, n: int):
    _check(load().lbm_step(ctx, n), ctx)


def lbm_step_save(ctx, state_ptr: int):
    _check(load().lbm_step_save(ctx, state_ptr), ctx)


def lbm_macros(ctx, rho_ptr, u_ptr, chi_ptr):
    _check(load().lbm_macros(ctx, rho_ptr, u_ptr, chi_ptr), ctx)


def lbm_diag(ctx, raise_unstable: bool = True) -> lbm_diagnostics:
    d = lbm_diagnostics()
    s = load().lbm_diag(ctx, C.byref(d))
    if s == LBM_ERR_UNSTABLE and not raise_unstable:
        return d
    _check(s, ctx)
    return d


def lbm_fw_accumulate(ctx, acc_ptr: int, weight: float):
    _check(load().lbm_fw_accumulate(ctx, acc_ptr, weight), ctx)


def lbm_get_state(ctx, dst_ptr: int):
    _check(load().lbm_get_state(ctx, dst_ptr), ctx)


def lbm_set_state(ctx, src_ptr: int, step: int):
    _check(load().lbm_set_state(ctx, src_ptr, step), ctx)


def lbm_adjoint_step(ctx, state_ptr, lam_next_ptr, lam_ptr, dcs_ptr, w_fw: float):
    _check(load().lbm_adjoint_step(ctx, state_ptr, lam_next_ptr, lam_ptr, dcs_ptr, w_fw), ctx)


def lbm_objective_forward(ctx, nsteps: int, K: int, ckpt_ptr, J_ptr):
    _check(load().lbm_objective_forward(ctx, nsteps, K, ckpt_ptr, J_ptr), ctx)


def lbm_adjoint_segment(ctx, ckpt_ptr, n0: int, k: int, seg_ptr, lam_ptr, tmp_ptr, dcs_ptr,
                        w_fw: float = 1.0):
    _check(load().lbm_adjoint_segment(ctx, ckpt_ptr, n0, k, seg_ptr, lam_ptr, tmp_ptr, dcs_ptr,
                                      w_fw), ctx)


def lbm_recompute_segment(ctx, ckpt_ptr, k: int, seg_ptr, stream=None):
    _check(load().lbm_recompute_segment(ctx, ckpt_ptr, k, seg_ptr, stream), ctx)


def lbm_adjoint_sweep(ctx, ckpt_ptr, seg_ptr, n0: int, k: int, lam_ptr, tmp_ptr, dcs_ptr,
                      w_fw: float = 1.0, stream=None):
    _check(load().lbm_adjoint_sweep(ctx, ckpt_ptr, seg_ptr, n0, k, lam_ptr, tmp_ptr, dcs_ptr, w_fw,
                                    stream), ctx)


def lbm_front_adjoint(ctx, state_ptr, lam_ptr, front_ptr):
    _check(load().lbm_front_adjoint(ctx, state_ptr, lam_ptr, front_ptr), ctx)


def lbm_adjoint_chi0(ctx, lam0_ptr, grad_ptr):
    _check(load().lbm_adjoint_chi0(ctx, lam0_ptr, grad_ptr), ctx)


def lbm_halo_bytes(p: lbm_params) -> int:
    return load().lbm_halo_bytes(C.byref(p))


def lbm_halo_pack(ctx, face: int, buf_ptr: int):
    _check(load().lbm_halo_pack(ctx, face, buf_ptr), ctx)


def lbm_halo_unpack(ctx, face: int, buf_ptr: int):
    _check(load().lbm_halo_unpack(ctx, face, buf_ptr), ctx)


def lbm_next_step_odd(ctx) -> int:
    return load().lbm_next_step_odd(ctx)


def lbm_column_max(ctx, m_ptr: int):
    _check(load().lbm_column_max(ctx, m_ptr), ctx)


def lbm_front_of_columns(m_ptr: int, nx: int, threshold: float, x0: int, H: int,
                         periodic_x: bool, out_ptr: int, stream_handle=None):
    _check(load().lbm_front_of_columns(m_ptr, nx, threshold, x0, H, int(periodic_x), out_ptr,
                                       stream_handle))


def lbm_get_step(ctx) -> int:
    return load().lbm_get_step(ctx)


def lbm_sync(ctx):
    _check(load().lbm_sync(ctx), ctx)


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def lbm_debug_build() -> bool:
    return bool(load().lbm_debug_build())


def lbm_debug_record(ctx) -> list[int]:
    """[failed checks, site of the first, its element offset, the extent checked]."""
    out = (C.c_int64 * 4)()
    _check(load().lbm_debug_record(ctx, out), ctx)
    return list(out)


# Index-check failures of the debug build over every Lattice destroyed so far
# in this process: [failed checks, first site, its offset, its extent].
DEBUG_TOTAL = [0, 0, 0, 0]


# --- parameters -----------------------------------------------------------------

@dataclass
class Params:
    """Mirror of lbm_params with the lock-exchange defaults of Sec. 2.5."""
    nx: int
    ny: int
    nz: int
    model: int = LBM_BGK_SMAG_Q19
    storage: int = LBM_FP32
    flags: int = 0
    nu: float = 8e-4
    D: float = 8e-4
    cs_smag: float = 0.17
    sc_t: float = 1.0
    gprime: float = 0.0
    eg: tuple = (0.0, 0.0, -1.0)
    omega_bulk: float = 1.0
    x0: int = 0
    H: int = 1
    noise_amp: float = 1e-3
    seed: int = 2112
    front_threshold: float = 0.02
    scale_f: float = 2.0 ** 14
    scale_phi: float = 2.0 ** 14
    scalar: int = LBM_SCALAR_Q7
    x_offset: int = 0          # x-slab: global x of local column 0
    nx_global: int = 0         # x-slab: nx of the whole box (0: a whole box)

    def c(self) -> lbm_params:
        p = lbm_params()
        for f in fields(self):
            v = getattr(self, f.name)
            if f.name == "eg":
                p.eg = (C.c_double * 3)(*v)
            else:
                setattr(p, f.name, v)
        return p

    @property
    def Q(self) -> int:
        return 27 if self.model == LBM_CUMULANT_Q27 else 19

    @property
    def NS(self) -> int:
        return {LBM_SCALAR_Q7: 7, LBM_SCALAR_Q6: 6, LBM_SCALAR_Q27: 27}[self.scalar]

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


GEOMETRIES = ("walls", "periodic")


def lock_exchange(nx: int, ny: int, nz: int, *, H: int, x0: int, u_b: float, Re: float,
                  Sc: float = 1.0, model: str = "bgk", storage: str = "fp32",
                  cs_smag: float = 0.17, scalar: str = "q7", geometry: str = "walls",
                  sc_t: float | str = 1.0, **kw) -> Params:
    """Lattice-unit parameters of the lock-exchange box (Sec. 2.5): g' = u_b^2 / H
    (u_b = sqrt(g' H)), nu = u_b H / Re_b, D = nu / Sc (Eq. 12-14).

    geometry: "walls" (Fig. 4a, Cases 2, 4, 6, 8: walls at the x ends) or
    "periodic" (Fig. 4b, Cases 1, 3, 5, 7: periodic ends; the span is periodic
    in both).  sc_t: turbulent Schmidt number of the BGK model's eddy
    diffusivity (Eq. 35), or "paper" for the literal Sc_T = C_s^2."""
    if geometry not in GEOMETRIES:
        raise ValueError(f"geometry must be one of {GEOMETRIES}")
    nu = u_b * H / Re
    flags = kw.pop("flags", 0) | (LBM_FLAG_PERIODIC_X if geometry == "periodic" else 0)
    sct = cs_smag * cs_smag if sc_t == "paper" else float(sc_t)
    return Params(nx=nx, ny=ny, nz=nz, model=MODELS[model], storage=STORAGES[storage],
                  nu=nu, D=nu / Sc, cs_smag=cs_smag, gprime=u_b * u_b / H, x0=x0, H=H,
                  scalar=SCALARS[scalar], flags=flags, sc_t=sct, **kw)


# --- torch-backed context -----------------------------------------------------------

class Lattice:
    """A context over a torch-allocated workspace on one CUDA device.

    All work goes to ``stream`` (default: torch's current stream).
    """

    def __init__(self, params: Params, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.params = params
        self._p = params.c()
        nbytes = lbm_workspace_bytes(self._p)
        if nbytes == 0:
            _check(lbm_validate(self._p))
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = lbm_init(self._p, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and _lib is not None:
            if _lib.lbm_debug_build():
                out = (C.c_int64 * 4)()
                if _lib.lbm_debug_record(ctx, out) == LBM_OK and out[0]:
                    if DEBUG_TOTAL[0] == 0:
                        DEBUG_TOTAL[1:] = list(out)[1:]
                    DEBUG_TOTAL[0] += out[0]
            _lib.lbm_destroy(ctx)
            self.ctx = None

    def debug_record(self) -> list[int]:
        return lbm_debug_record(self.ctx)

    @property
    def Q(self) -> int:
        return self.params.Q

    @property
    def NS(self) -> int:
        return self.params.NS

    @property
    def N(self) -> int:
        return self.params.N

    def _empty(self, *shape, dtype=None):
        return self.torch.empty(*shape, dtype=dtype or self.torch.float32, device=self.device)

    def set_scalar(self, chi0):
        """chi0: float32 tensor of N values (host or device)."""
        assert chi0.dtype == self.torch.float32 and chi0.numel() == self.N and chi0.is_contiguous()
        lbm_set_scalar(self.ctx, chi0.data_ptr())

    def step(self, n: int = 1):
        lbm_step(self.ctx, n)

    def step_save(self, out):
        lbm_step_save(self.ctx, out.data_ptr())

    def macros(self):
        rho = self._empty(self.N)
        u = self._empty(3, self.N)
        chi = self._empty(self.N)
        lbm_macros(self.ctx, rho.data_ptr(), u.data_ptr(), chi.data_ptr())
        sh = self.params.shape
        return rho.view(sh), u.view((3,) + sh), chi.view(sh)

    def diag(self, raise_unstable: bool = True) -> dict:
        return lbm_diag(self.ctx, raise_unstable).as_dict()

    def fw_accumulate(self, acc, weight: float = 1.0):
        lbm_fw_accumulate(self.ctx, acc.data_ptr(), weight)

    def get_state(self, out=None):
        if out is None:
            out = self._empty(self.Q + self.NS, self.N)
        lbm_get_state(self.ctx, out.data_ptr())
        return out

    def set_state(self, src, step: int = 0):
        assert (src.dtype == self.torch.float32 and src.is_contiguous()
                and src.numel() == (self.Q + self.NS) * self.N)
        lbm_set_state(self.ctx, src.data_ptr(), step)

    def adjoint_step(self, state, lam_next, lam, dcs, w_fw: float):
        lbm_adjoint_step(self.ctx, state.data_ptr(), _ptr(lam_next), lam.data_ptr(),
                         dcs.data_ptr() if dcs is not None else None, w_fw)

    def objective_forward(self, nsteps: int, K: int, ckpt, acc):
        lbm_objective_forward(self.ctx, nsteps, K, _ptr(ckpt), _ptr(acc))

    def adjoint_segment(self, ckpt, n0: int, k: int, seg, lam, tmp, dcs, w_fw: float = 1.0):
        lbm_adjoint_segment(self.ctx, ckpt.data_ptr(), n0, k, _ptr(seg), lam.data_ptr(),
                            tmp.data_ptr(), dcs.data_ptr() if dcs is not None else None, w_fw)

    def recompute_segment(self, ckpt, k: int, seg, stream=None):
        """States n0+1 .. n0+k-1 from the checkpoint into seg[1 .. k-1] on
        `stream` (a torch.cuda.Stream; None: the lattice's stream)."""
        lbm_recompute_segment(self.ctx, ckpt.data_ptr(), k, _ptr(seg),
                              stream.cuda_stream if stream is not None else None)

    def adjoint_sweep(self, ckpt, seg, n0: int, k: int, lam, tmp, dcs, w_fw: float = 1.0,
                      stream=None):
        """k reverse steps through ckpt and seg on `stream` (None: the
        lattice's stream)."""
        lbm_adjoint_sweep(self.ctx, ckpt.data_ptr(), _ptr(seg), n0, k, lam.data_ptr(),
                          tmp.data_ptr(), dcs.data_ptr() if dcs is not None else None, w_fw,
                          stream.cuda_stream if stream is not None else None)

    def front_adjoint(self, state, lam=None, value=None):
        """Front of `state` (canonical layout) into `value` (one device double)
        and its derivative into `lam`; either may be None."""
        lbm_front_adjoint(self.ctx, state.data_ptr(), _ptr(lam), _ptr(value))

    def adjoint_chi0(self, lam0, grad):
        lbm_adjoint_chi0(self.ctx, lam0.data_ptr(), grad.data_ptr())

    def halo_pack(self, face: int, buf):
        lbm_halo_pack(self.ctx, face, buf.data_ptr())

    def halo_unpack(self, face: int, buf):
        lbm_halo_unpack(self.ctx, face, buf.data_ptr())

    @property
    def next_step_odd(self) -> bool:
        return lbm_next_step_odd(self.ctx) == 1

    def column_max(self, out=None):
        """m(x) = max over z of the span-averaged chi, one float per column."""
        if out is None:
            out = self._empty(self.params.nx)
        lbm_column_max(self.ctx, out.data_ptr())
        return out

    def front_of_columns(self, m, nx: int, threshold: float, x0: int, H: int,
                         periodic_x: bool):
        """Front of a whole box from its column maxima m (device, nx floats):
        (value, node coordinate) as in diag()."""
        out = self._empty(2, dtype=self.torch.float64)
        lbm_front_of_columns(m.data_ptr(), nx, threshold, x0, H, periodic_x, out.data_ptr(),
                             self.stream.cuda_stream)
        v = out.cpu()
        return float(v[0]), float(v[1])

    @property
    def step_count(self) -> int:
        return lbm_get_step(self.ctx)

    def sync(self):
        lbm_sync(self.ctx)
