"""ctypes view of the plain FP64 C oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy
float64, node-major array-of-structures: ``f`` has shape (nz, ny, nx, Q),
``phi`` (nz, ny, nx, 7), macros (nz, ny, nx) and u (nz, ny, nx, 3).

Each wrapper cites the passage of the paper its C function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

__all__ = [
    "OracleParams", "build", "lib", "q_of", "velocities", "velocities_q7",
    "feq_q19", "phieq_q7", "tau_eff", "collide_node", "cumulants27",
    "f_from_cumulants27", "bgk_nu_t", "lock_chi0", "init", "step", "run", "stream",
    "macros", "wall_friction", "front_node", "diag", "splitmix64", "velocities_scalar",
    "phieq_q6", "front_xlim", "set_threads", "threads", "run_inplace",
]


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (IEEE arithmetic, no fast-math), with
    OpenMP for the node loops where the compiler has it (the arithmetic and
    its order per node are the same with and without)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


class _P(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("model", C.c_int), ("periodic_x", C.c_int), ("periodic_z", C.c_int),
                ("no_collide", C.c_int), ("pad_", C.c_int),
                ("nu", C.c_double), ("D", C.c_double), ("cs_smag", C.c_double),
                ("sc_t", C.c_double), ("gprime", C.c_double), ("eg", C.c_double * 3),
                ("omega_bulk", C.c_double), ("omega_high", C.c_double),
                ("scalar", C.c_int), ("pad2_", C.c_int), ("omega_phi_high", C.c_double)]


@dataclass
class OracleParams:
    nx: int
    ny: int
    nz: int
    model: int = 0            # 0 BGK-Smagorinsky D3Q19, 1 cumulant D3Q27
    nu: float = 8e-4
    D: float = 8e-4
    cs_smag: float = 0.17
    sc_t: float = 1.0
    gprime: float = 0.0
    eg: tuple = (0.0, 0.0, -1.0)
    omega_bulk: float = 1.0
    omega_high: float = 1.0
    periodic_x: bool = False
    periodic_z: bool = False
    no_collide: bool = False
    scalar: int = 0           # 0 D3Q7 BGK, 1 D3Q6 BGK, 2 D3Q27 factorized central moments
    omega_phi_high: float = 1.0
    _c: _P = field(default=None, repr=False)

    def c(self) -> _P:
        p = _P()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.model = self.model
        p.periodic_x, p.periodic_z = int(self.periodic_x), int(self.periodic_z)
        p.no_collide = int(self.no_collide)
        p.nu, p.D, p.cs_smag, p.sc_t, p.gprime = self.nu, self.D, self.cs_smag, self.sc_t, self.gprime
        p.eg = (C.c_double * 3)(*self.eg)
        p.omega_bulk, p.omega_high = self.omega_bulk, self.omega_high
        p.scalar, p.omega_phi_high = self.scalar, self.omega_phi_high
        return p

    @property
    def Q(self) -> int:
        return 27 if self.model == 1 else 19

    @property
    def NS(self) -> int:
        return {0: 7, 1: 6, 2: 27}[self.scalar]

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        i = C.POINTER(C.c_int)
        P = C.POINTER(_P)
        sig = {
            "orc_q": (C.c_int, [C.c_int]),
            "orc_velocities": (None, [C.c_int, i, d]),
            "orc_velocities_q7": (None, [i, d]),
            "orc_ns": (C.c_int, [C.c_int]),
            "orc_velocities_scalar": (None, [C.c_int, i, d]),
            "orc_phieq_q6": (None, [C.c_double, d, d]),
            "orc_feq_q19": (None, [C.c_double, d, d]),
            "orc_phieq_q7": (None, [C.c_double, d, d]),
            "orc_tau_eff": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_cumulants27": (None, [d, d]),
            "orc_f_from_cumulants27": (None, [d, d]),
            "orc_collide_node": (None, [P, d, d, d, d]),
            "orc_bgk_nu_t": (C.c_double, [P, d, d]),
            "orc_stream": (None, [P, d, d, d, d]),
            "orc_macros": (None, [P, d, d, d, d, d]),
            "orc_wall_friction": (C.c_double, [C.c_int, C.c_int, C.c_int, C.c_double, d]),
            "orc_front_node": (C.c_double, [C.c_int, C.c_int, C.c_int, d, C.c_double]),
            "orc_front_node_lim": (C.c_double, [C.c_int, C.c_int, C.c_int, d, C.c_double, C.c_int]),
            "orc_front_xlim": (C.c_int, [C.c_int, C.c_int, C.c_int]),
            "orc_diag": (None, [P, d, d, C.c_int, C.c_double, C.c_double, d]),
            "orc_step": (None, [P, d, d]),
            "orc_run": (None, [P, C.c_int, d, d, d]),
            "orc_splitmix64": (C.c_uint64, [C.c_uint64]),
            "orc_lock_chi0": (None, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64, d]),
            "orc_init": (None, [P, d, d, d]),
            "orc_set_threads": (C.c_int, [C.c_int]),
            "orc_threads": (C.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> int:
    """Threads of the node loops (1 = the plain serial oracle); returns the
    count in effect (1 when built without OpenMP).  Results do not depend on
    it: each node is computed on its own and the reductions stay serial."""
    return lib().orc_set_threads(int(n))


def threads() -> int:
    return lib().orc_threads()


def q_of(model: int) -> int:
    return lib().orc_q(model)


def velocities(model: int):
    """Velocity set and weights: D3Q19 (Eq. 23-24) or D3Q27 (Eq. 36)."""
    q = q_of(model)
    c = np.zeros(3 * q, dtype=np.int32)
    w = np.zeros(q)
    lib().orc_velocities(model, c.ctypes.data_as(C.POINTER(C.c_int)), _d(w))
    return c.reshape(q, 3), w


def velocities_q7():
    """D3Q7 scalar lattice (reading R1: w0 = 1/4, w = 1/8)."""
    c = np.zeros(21, dtype=np.int32)
    w = np.zeros(7)
    lib().orc_velocities_q7(c.ctypes.data_as(C.POINTER(C.c_int)), _d(w))
    return c.reshape(7, 3), w


def velocities_scalar(scalar: int):
    """Scalar lattice: D3Q7 (R1), D3Q6 (Eq. 31, w = 1/6) or D3Q27 (Eq. 36)."""
    n = lib().orc_ns(scalar)
    c = np.zeros(3 * n, dtype=np.int32)
    w = np.zeros(n)
    lib().orc_velocities_scalar(scalar, c.ctypes.data_as(C.POINTER(C.c_int)), _d(w))
    return c.reshape(n, 3), w


def phieq_q6(chi: float, u) -> np.ndarray:
    """Scalar equilibrium, Eq. 29 on D3Q6 (c_s^2 = 1/3)."""
    out = np.zeros(6)
    lib().orc_phieq_q6(chi, _d(_f64(u)), _d(out))
    return out


def feq_q19(rho: float, u) -> np.ndarray:
    """Second-order equilibrium, Eq. 22."""
    out = np.zeros(19)
    lib().orc_feq_q19(rho, _d(_f64(u)), _d(out))
    return out


def phieq_q7(chi: float, u) -> np.ndarray:
    """Scalar equilibrium, Eq. 29 on D3Q7."""
    out = np.zeros(7)
    lib().orc_phieq_q7(chi, _d(_f64(u)), _d(out))
    return out


def tau_eff(tau0: float, cs: float, q: float, rho: float) -> float:
    """Smagorinsky relaxation time, closed form of Eq. 34 (reading R3)."""
    return lib().orc_tau_eff(tau0, cs, q, rho)


def collide_node(p: OracleParams, f, phi):
    """Fluid + scalar collision at one node (Eq. 17-35)."""
    f = _f64(f)
    phi = _f64(phi)
    fo = np.zeros(p.Q)
    po = np.zeros(p.NS)
    pc = p.c()
    lib().orc_collide_node(C.byref(pc), _d(f), _d(phi), _d(fo), _d(po))
    return fo, po


def bgk_nu_t(p: OracleParams, f, phi) -> float:
    """Eddy viscosity of the BGK-Smagorinsky collision at one node (Eq. 32-34)."""
    pc = p.c()
    return lib().orc_bgk_nu_t(C.byref(pc), _d(_f64(f)), _d(_f64(phi)))


def cumulants27(f) -> np.ndarray:
    """Cumulants C_abc (Eq. 54) for a, b, c <= 2; index (a*3+b)*3+c; C[0] = ln rho."""
    out = np.zeros(27)
    lib().orc_cumulants27(_d(_f64(f)), _d(out))
    return out


def f_from_cumulants27(Cs) -> np.ndarray:
    out = np.zeros(27)
    lib().orc_f_from_cumulants27(_d(_f64(Cs)), _d(out))
    return out


def splitmix64(s: int) -> int:
    return int(lib().orc_splitmix64(s & 0xFFFFFFFFFFFFFFFF))


def lock_chi0(nx, ny, nz, x0, amp=1e-3, seed=2112) -> np.ndarray:
    """Lock-exchange initial scalar (Table 1, Sec. 2.5; noise reading R10)."""
    out = np.zeros((nz, ny, nx))
    lib().orc_lock_chi0(nx, ny, nz, x0, amp, seed, _d(out))
    return out


def init(p: OracleParams, chi0):
    """Rest state f = w, Phi = w chi0."""
    chi0 = _f64(chi0).reshape(p.shape)
    f = np.zeros(p.shape + (p.Q,))
    phi = np.zeros(p.shape + (p.NS,))
    pc = p.c()
    lib().orc_init(C.byref(pc), _d(chi0), _d(f), _d(phi))
    return f, phi


def step(p: OracleParams, f, phi):
    """One time step (collide, then stream) in place on copies; returns them."""
    f = _f64(f).copy()
    phi = _f64(phi).copy()
    pc = p.c()
    lib().orc_step(C.byref(pc), _d(f), _d(phi))
    return f, phi


def run(p: OracleParams, nsteps: int, f, phi, record_fw: bool = False):
    """nsteps time steps; optionally F_w after every step."""
    f = _f64(f).copy()
    phi = _f64(phi).copy()
    fw = np.zeros(max(nsteps, 1)) if record_fw else None
    pc = p.c()
    lib().orc_run(C.byref(pc), nsteps, _d(f), _d(phi), _d(fw) if fw is not None else None)
    if record_fw:
        return f, phi, fw[:nsteps]
    return f, phi


def run_inplace(p: OracleParams, nsteps: int, f: np.ndarray, phi: np.ndarray) -> None:
    """nsteps time steps on the caller's arrays (float64, C-contiguous), no
    copies: for timing large boxes."""
    pc = p.c()
    lib().orc_run(C.byref(pc), nsteps, _d(f), _d(phi), None)


def stream(p: OracleParams, fpost, phipost):
    """Streaming only (pull form of Eq. 17, half-way bounce-back)."""
    fpost = _f64(fpost)
    phipost = _f64(phipost)
    f = np.zeros_like(fpost)
    phi = np.zeros_like(phipost)
    pc = p.c()
    lib().orc_stream(C.byref(pc), _d(fpost), _d(phipost), _d(f), _d(phi))
    return f, phi


def macros(p: OracleParams, f, phi):
    """rho (Eq. 19), u with the half-force shift (Eq. 20), chi (Eq. 27)."""
    f = _f64(f)
    phi = _f64(phi)
    rho = np.zeros(p.shape)
    u = np.zeros(p.shape + (3,))
    chi = np.zeros(p.shape)
    pc = p.c()
    lib().orc_macros(C.byref(pc), _d(f), _d(phi), _d(rho), _d(u), _d(chi))
    return rho, u, chi


def wall_friction(nu: float, u) -> float:
    """F_w (Eq. 64) from tau_w (Eq. 62) by the one-sided quadratic (reading R12)."""
    u = _f64(u)
    nz, ny, nx, _ = u.shape
    return lib().orc_wall_friction(nx, ny, nz, nu, _d(u))


def front_node(chi, thr: float = 0.02, xlim: int | None = None) -> float:
    """Front node coordinate from the span-averaged field (Sec. 3.1, R11),
    searching the columns x < xlim (default all)."""
    chi = _f64(chi)
    nz, ny, nx = chi.shape
    return lib().orc_front_node_lim(nx, ny, nz, _d(chi), thr, nx if xlim is None else xlim)


def front_xlim(nx: int, x0: int, periodic_x: bool) -> int:
    """Columns searched for the front: nx, or (nx + x0) // 2 with periodic ends."""
    return lib().orc_front_xlim(nx, x0, int(bool(periodic_x)))


def diag(p: OracleParams, f, phi, x0: int, H: float, thr: float = 0.02) -> dict:
    out = np.zeros(5)
    pc = p.c()
    lib().orc_diag(C.byref(pc), _d(_f64(f)), _d(_f64(phi)), x0, H, thr, _d(out))
    return {"front": out[0], "Fw": out[1], "mass_delta": out[2], "scalar_mass": out[3],
            "front_node": out[4]}
