"""FP64 CPU oracle of the particle stochastic-Galerkin Boltzmann scheme (arXiv:2404.19602).

TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package.  It shares no code with the CUDA library; both read the
same seeded workload descriptions (plain parameter dictionaries) and each implements Philox
itself.

The numerics live in ``pgc_oracle.c`` (plain C, FP64, OpenMP over particles as Remark 1 of
Sec. 3 allows); this module only builds it with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpgc_oracle.so")
_lock = threading.Lock()
_lib = None

# mechanism bits (order of the rate vector of Eq. (20))
AC, OPM, OPP, KM, KP, EDGE = 1, 2, 4, 8, 16, 32
ALL_MECH = 63
PAULI_INITIAL_MAX, PAULI_CURRENT_MAX, PAULI_OFF = 0, 1, 2
FS_PAPER, FS_EXACT_ENERGY = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction so that x86 and Arm agree bit for bit)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [
        ("T_K", C.c_double), ("eps_F", C.c_double),
        ("eps0_lo", C.c_double), ("eps0_hi", C.c_double),
        ("Ex_lo", C.c_double), ("Ex_hi", C.c_double),
        ("mech_mask", C.c_uint32), ("alpha", C.c_double),
        ("Nk", C.c_int32), ("Lk_hvF", C.c_double),
        ("M", C.c_int32), ("Q1", C.c_int32),
        ("N", C.c_int64), ("dt_fs", C.c_double),
        ("seed", C.c_uint64), ("stream_id", C.c_uint32),
        ("pauli_norm", C.c_int32), ("final_state", C.c_int32),
        ("n_theta", C.c_int32), ("max_coll", C.c_int32),
        ("eps0_law", C.c_int32), ("W_lo", C.c_double), ("W_hi", C.c_double),
        ("splitting", C.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, dp, u32p, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_uint32), C.POINTER(C.c_int64)
            L.orc_create.restype = vp
            L.orc_create.argtypes = [C.POINTER(_Cfg)]
            L.orc_destroy.argtypes = [vp]
            L.orc_init.argtypes = [vp, dp]
            L.orc_step.argtypes = [vp, C.c_int64, C.c_int64]
            L.orc_sizes.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.orc_get_state.argtypes = [vp, dp]
            L.orc_set_state.argtypes = [vp, dp]
            L.orc_get_hist.argtypes = [vp, u32p, u32p]
            L.orc_get_tables.argtypes = [vp] + [dp] * 8
            L.orc_get_constants.argtypes = [vp, dp]
            L.orc_get_counters.argtypes = [vp, i64p]
            L.orc_num_outputs.restype = C.c_int64
            L.orc_num_outputs.argtypes = [vp]
            L.orc_get_moments.argtypes = [vp, dp, dp, dp, dp]
            L.orc_reconstruct_f.argtypes = [vp, dp, C.c_int, u32p, u32p]
            L.orc_observe_at.argtypes = [vp, dp, dp]
            L.orc_rates.argtypes = [vp, C.c_double, C.c_double, C.c_double, dp]
            L.orc_philox.argtypes = [u32p, u32p, u32p]
            L.orc_u01.restype = C.c_double
            L.orc_u01.argtypes = [C.c_uint32]
            L.orc_li2_neg.restype = C.c_double
            L.orc_li2_neg.argtypes = [C.c_double]
            L.orc_fd_total.restype = C.c_double
            L.orc_fd_total.argtypes = [C.c_double] * 3
            L.orc_fd_sample.restype = C.c_double
            L.orc_fd_sample.argtypes = [C.c_double] * 4
            L.orc_gauss_legendre.argtypes = [C.c_int, dp, dp]
            L.orc_psi_at.argtypes = [C.POINTER(_Cfg), dp, dp]
            L.orc_edge_T.restype = C.c_double
            L.orc_edge_T.argtypes = [C.c_double, C.c_double, C.c_int]
            L.orc_angle_edge.restype = C.c_double
            L.orc_angle_edge.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
            L.orc_angle_ac.restype = C.c_double
            L.orc_angle_ac.argtypes = [C.c_double]
            L.orc_angle_k.restype = C.c_double
            L.orc_angle_k.argtypes = [C.c_double]
            L.orc_project_nodes.argtypes = [vp, dp, dp]
            L.orc_recon_nodes.argtypes = [vp, dp, dp]
            L.orc_tangent_run.restype = C.c_int
            L.orc_tangent_run.argtypes = [vp, C.c_int64, C.c_int64, C.c_int64, dp, dp]
            L.orc_window_objective.restype = C.c_int
            L.orc_window_objective.argtypes = [vp, C.c_int64, C.c_int64, C.c_int64, dp]
            L.orc_step_particles.argtypes = [vp, i64p, C.c_int64]
            L.orc_set_step.argtypes = [vp, C.c_int64]
            L.orc_set_nmax.argtypes = [vp, u32p]
            L.orc_set_hist.argtypes = [vp, u32p]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


DEFAULTS = dict(T_K=300.0, eps_F=0.4, eps0_lo=0.1, eps0_hi=0.1, Ex_lo=5000.0, Ex_hi=5000.0,
                mech_mask=ALL_MECH, alpha=0.1, Nk=240, Lk_hvF=5.0, M=5, Q1=6, N=1000,
                dt_fs=1.0, seed=1, stream_id=0, pauli_norm=PAULI_INITIAL_MAX,
                final_state=FS_PAPER, n_theta=64, max_coll=32, eps0_law=0, W_lo=0.0, W_hi=0.0,
                splitting=0)


def make_cfg(params: dict) -> _Cfg:
    p = dict(DEFAULTS)
    for k, v in params.items():
        if k in p:
            p[k] = v
    if (params.get("W_lo") or 0.0) > 0.0:   # the width is the input: eps0 = pi hbar vF / W
        p["eps0_law"] = 1
        p["W_hi"] = params.get("W_hi", params["W_lo"])
    c = _Cfg()
    for k, v in p.items():
        setattr(c, k, v)
    return c


# ---------------------------------------------------------------------------------------------
# elementary functions (for the pins)
# ---------------------------------------------------------------------------------------------
def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_u32p(c), _u32p(k), _u32p(o))
    return o


def u01(x):
    return lib().orc_u01(int(x))


def li2_neg(x):
    return lib().orc_li2_neg(float(x))


def fd_total(eps0, mu, kT):
    return lib().orc_fd_total(eps0, mu, kT)


def fd_sample(eps0, mu, kT, u):
    return lib().orc_fd_sample(eps0, mu, kT, u)


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def edge_T(beta, c, n=64):
    return lib().orc_edge_T(beta, c, n)


def angle_edge(beta, c, u, n=64):
    return lib().orc_angle_edge(beta, c, u, n)


def angle_ac(u):
    return lib().orc_angle_ac(u)


def angle_k(u):
    return lib().orc_angle_k(u)


def num_threads():
    return lib().orc_num_threads()


def set_threads(n: int):
    """Threads of the oracle's parallel loops (n <= 0: all host cores)."""
    lib().orc_set_threads(int(n))


class Oracle:
    """One ensemble of N particles advanced by the oracle.

    State layout: khat[c][h][i] (c = x,y; h = gPC coefficient in graded order; i = particle),
    float64, the same layout the CUDA library's pgc_get_state returns.
    """

    def __init__(self, params: dict, init_khat: np.ndarray | None = None):
        self.params = dict(DEFAULTS)
        self.params.update({k: v for k, v in params.items() if k in DEFAULTS})
        self._cfg = make_cfg(self.params)
        L = lib()
        self._h = L.orc_create(C.byref(self._cfg))
        d, P, Q = C.c_int(), C.c_int(), C.c_int()
        L.orc_sizes(self._h, C.byref(d), C.byref(P), C.byref(Q))
        self.d, self.P, self.Q = d.value, P.value, Q.value
        self.N = int(self.params["N"])
        self.Nk = int(self.params["Nk"])
        if init_khat is not None:
            a = np.ascontiguousarray(init_khat, dtype=np.float64).reshape(2, self.P, self.N)
            L.orc_init(self._h, _dp(a))
        else:
            L.orc_init(self._h, None)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def step(self, nsteps: int, moments_every: int = 10):
        lib().orc_step(self._h, int(nsteps), int(moments_every))

    def state(self) -> np.ndarray:
        a = np.zeros((2, self.P, self.N))
        lib().orc_get_state(self._h, _dp(a))
        return a

    def set_state(self, khat):
        a = np.ascontiguousarray(khat, dtype=np.float64).reshape(2, self.P, self.N)
        lib().orc_set_state(self._h, _dp(a))

    def hist(self):
        H = np.zeros((self.Q, self.Nk, self.Nk), dtype=np.uint32)
        m = np.zeros(self.Q, dtype=np.uint32)
        lib().orc_get_hist(self._h, _u32p(H), _u32p(m))
        return H, m

    def tables(self):
        Q, P, d = self.Q, self.P, self.d
        zq = np.zeros((Q, max(d, 1)))
        wq, eps0q, Exq, dq, nq = (np.zeros(Q) for _ in range(5))
        psi = np.zeros((Q, P))
        dhat = np.zeros(P)
        lib().orc_get_tables(self._h, _dp(zq), _dp(wq), _dp(psi), _dp(eps0q), _dp(Exq), _dp(dq),
                             _dp(nq), _dp(dhat))
        return dict(z=zq[:, :d] if d else zq[:, :0], w=wq, psi=psi, eps0=eps0q, Ex=Exq, d=dq, n=nq,
                    dhat=dhat)

    def constants(self):
        a = np.zeros(14)
        lib().orc_get_constants(self._h, _dp(a))
        keys = ["hvF", "hbar_fs", "kT", "Cac", "CO", "CK", "nO", "nK", "hwO", "hwK", "Cedg", "a_nm",
                "Lk", "dk"]
        return dict(zip(keys, a.tolist()))

    def counters(self):
        a = np.zeros(6, dtype=np.int64)
        lib().orc_get_counters(self._h, a.ctypes.data_as(C.POINTER(C.c_int64)))
        return dict(zip(["attempts", "real", "rejected", "capped", "out_of_grid", "step"], a.tolist()))

    def moments(self):
        L = lib()
        T = L.orc_num_outputs(self._h)
        t = np.zeros(T)
        nodes = np.zeros((T, self.Q, 4))
        mean = np.zeros((T, 4))
        var = np.zeros((T, 4))
        L.orc_get_moments(self._h, _dp(t), _dp(nodes), _dp(mean), _dp(var))
        return dict(t_fs=t, nodes=nodes, mean=mean, var=var)

    def rates(self, kx, ky, eps0):
        g = np.zeros(6)
        lib().orc_rates(self._h, float(kx), float(ky), float(eps0), _dp(g))
        return g

    def psi_at(self, z):
        z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.float64)
        out = np.zeros(self.P)
        lib().orc_psi_at(C.byref(self._cfg), _dp(z), _dp(out))
        return out

    def reconstruct_f(self, z):
        z = np.ascontiguousarray(np.asarray(z, dtype=np.float64).reshape(-1, max(self.d, 1)))
        nz = z.shape[0]
        H = np.zeros((nz, self.Nk, self.Nk), dtype=np.uint32)
        m = np.zeros(nz, dtype=np.uint32)
        lib().orc_reconstruct_f(self._h, _dp(z), nz, _u32p(H), _u32p(m))
        return H, m

    def project_nodes(self, vq):
        vq = np.ascontiguousarray(vq, dtype=np.float64)
        out = np.zeros(self.P)
        lib().orc_project_nodes(self._h, _dp(vq), _dp(out))
        return out

    def recon_nodes(self, vhat):
        vhat = np.ascontiguousarray(vhat, dtype=np.float64)
        out = np.zeros(self.Q)
        lib().orc_recon_nodes(self._h, _dp(vhat), _dp(out))
        return out

    def tangent_run(self, nsteps, every, window):
        """Pathwise sensitivities (events frozen) of the window averages of mean_z J_x and
        var_z J_x with respect to (E_lo, E_hi, eps0_lo, eps0_hi); advances the state."""
        val = np.zeros(2)
        grad = np.zeros(8)
        r = lib().orc_tangent_run(self._h, int(nsteps), int(every), int(window), _dp(val), _dp(grad))
        if r != 0:
            raise RuntimeError("orc_tangent_run failed (%d)" % r)
        return val, grad.reshape(2, 4)

    def window_objective(self, nsteps, every, window):
        val = np.zeros(2)
        r = lib().orc_window_objective(self._h, int(nsteps), int(every), int(window), _dp(val))
        if r != 0:
            raise RuntimeError("orc_window_objective failed (%d)" % r)
        return val

    def step_particles(self, idx):
        """Advance only the particles idx by one time step against the current histogram
        (test hook; the step counter and the histogram stay)."""
        a = np.ascontiguousarray(idx, dtype=np.int64)
        lib().orc_step_particles(self._h, a.ctypes.data_as(C.POINTER(C.c_int64)), a.size)

    def set_step(self, step):
        lib().orc_set_step(self._h, int(step))

    def set_nmax(self, nmax):
        a = np.ascontiguousarray(nmax, dtype=np.uint32)
        lib().orc_set_nmax(self._h, _u32p(a))

    def set_hist(self, H):
        """Replace the histogram f^n [Q][Nk][Nk] that the next step's Pauli test reads (test hook)."""
        a = np.ascontiguousarray(H, dtype=np.uint32).reshape(self.Q, self.Nk, self.Nk)
        lib().orc_set_hist(self._h, _u32p(a))

    def observe_at(self, z):
        z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.float64)
        out = np.zeros(4)
        lib().orc_observe_at(self._h, _dp(z), _dp(out))
        return out
