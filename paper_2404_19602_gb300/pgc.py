"""Thin Python binding of the C ABI in include/pgc.h (argument marshalling only).

The functions keep the C names (pgc_query_sizes, pgc_init, pgc_step, pgc_moments,
pgc_reconstruct_f, ...).  Every step of the particle scheme runs in the CUDA kernels of
libpgc.so; PyTorch only provides the caller-owned device buffers and the CUDA stream.  There is
no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpgc.so")
_lock = threading.Lock()
_lib = None

PGC_OK, PGC_EINVAL, PGC_ENOMEM, PGC_ECUDA, PGC_ESTATE, PGC_ETIMEOUT, PGC_EUNSUPPORTED = range(7)
PGC_FP32, PGC_FP64 = 0, 1
PGC_MECH_ALL = 63
COUNTER_NAMES = ["attempts", "changed", "rejected", "capped", "out_of_grid", "queued", "error", "steps"]


class PgcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


_STATUS = {0: "PGC_OK", 1: "PGC_EINVAL", 2: "PGC_ENOMEM", 3: "PGC_ECUDA", 4: "PGC_ESTATE",
           5: "PGC_ETIMEOUT", 6: "PGC_EUNSUPPORTED"}


class pgc_interval(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double)]


class pgc_config(C.Structure):
    _fields_ = [
        ("T_K", C.c_double), ("eps_F_eV", C.c_double),
        ("eps0_eV", pgc_interval), ("Ex_Vcm", pgc_interval),
        ("mech_mask", C.c_uint32), ("alpha", C.c_double),
        ("Nk", C.c_int32), ("Lk_hvF_eV", C.c_double),
        ("degree_M", C.c_int32), ("quad_per_dim", C.c_int32),
        ("n_particles", C.c_int64), ("dt_fs", C.c_double),
        ("seed", C.c_uint64), ("stream_id", C.c_uint32),
        ("precision", C.c_int32), ("pauli_norm", C.c_int32), ("final_state", C.c_int32),
        ("n_theta_edge", C.c_int32), ("max_collisions", C.c_int32), ("max_outputs", C.c_int32),
        ("eps0_law", C.c_int32), ("width_nm", pgc_interval), ("splitting", C.c_int32), ("tc_proj", C.c_int32),
    ]


PGC_EPS0_AFFINE, PGC_EPS0_WIDTH = 0, 1
PGC_SPLIT_LIE, PGC_SPLIT_STRANG = 0, 1
PGC_TC_OFF, PGC_TC_F16X3, PGC_TC_F16 = 0, 1, 2


_vp, _dp, _u32p, _u64p, _i64p = (C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_uint32),
                                 C.POINTER(C.c_uint64), C.POINTER(C.c_int64))

#: exported symbols with (restype, argtypes); the header declares exactly these
SIGNATURES = {
    "pgc_config_default": (None, [C.POINTER(pgc_config)]),
    "pgc_query_sizes": (C.c_int, [C.POINTER(pgc_config), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                  C.POINTER(C.c_size_t), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pgc_init": (C.c_int, [C.POINTER(pgc_config), _vp, _vp, _vp, _dp, _vp, C.POINTER(_vp)]),
    "pgc_step": (C.c_int, [_vp, C.c_int64, C.c_int32]),
    "pgc_set_pipeline": (C.c_int, [_vp, C.c_int32]),
    "pgc_moments": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _i64p]),
    "pgc_reconstruct_f": (C.c_int, [_vp, _dp, C.c_int32, _u32p, _u32p]),
    "pgc_observe_at": (C.c_int, [_vp, _dp, C.c_int32, _dp]),
    "pgc_get_state": (C.c_int, [_vp, _dp]),
    "pgc_set_state": (C.c_int, [_vp, _dp]),
    "pgc_get_state_native": (C.c_int, [_vp, _vp]),
    "pgc_set_state_native": (C.c_int, [_vp, _vp]),
    "pgc_counters": (C.c_int, [_vp, _u64p]),
    "pgc_get_hist": (C.c_int, [_vp, _u32p, _u32p]),
    "pgc_profile": (C.c_int, [_vp, C.c_int32]),
    "pgc_profile_read": (C.c_int, [_vp, _dp, _dp, _i64p]),
    "pgc_profile_timeline": (C.c_int, [_vp, _dp, C.c_int64, _i64p]),
    "pgc_observe_static": (C.c_int, [_vp, _vp, _vp, _vp]),
    "pgc_batch_query_sizes": (C.c_int, [C.POINTER(_vp), C.c_int32, C.POINTER(C.c_size_t)]),
    "pgc_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int32, _vp, C.c_int32, C.POINTER(_vp)]),
    "pgc_batch_step": (C.c_int, [_vp, C.c_int64, C.c_int32, C.c_int32]),
    "pgc_batch_autotune": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32), _dp]),
    "pgc_batch_destroy": (None, [_vp]),
    "pgc_window_objective": (C.c_int, [_vp, C.c_int64, C.c_int32, C.c_int64, _dp]),
    "pgc_batch_launch_config": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "pgc_batch_last_error": (C.c_char_p, [_vp]),
    "pgc_adjoint_query_sizes": (C.c_int, [_vp, C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]),
    "pgc_adjoint": (C.c_int, [_vp, C.c_int64, C.c_int32, C.c_int32, C.c_int64, _dp, _vp, _dp, _dp]),
    "pgc_destroy": (None, [_vp]),
    "pgc_last_error": (C.c_char_p, [_vp]),
    "pgc_status_string": (C.c_char_p, [C.c_int]),
    "pgc_launch_count": (C.c_uint64, []),
}


def lib():
    """Load libpgc.so (built by paper_2404_19602_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libpgc.so not built (%s); run paper_2404_19602_gb300.build.build()" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status, ctx=None):
    if status != PGC_OK:
        msg = lib().pgc_last_error(ctx)
        raise PgcError(status, msg.decode() if msg else "")


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


# ------------------------------------------------------------------------------------------
# same-name wrappers
# ------------------------------------------------------------------------------------------
def pgc_config_default() -> pgc_config:
    c = pgc_config()
    lib().pgc_config_default(C.byref(c))
    return c


def pgc_query_sizes(cfg: pgc_config):
    s, h, x = C.c_size_t(), C.c_size_t(), C.c_size_t()
    P, Q = C.c_int32(), C.c_int32()
    _check(lib().pgc_query_sizes(C.byref(cfg), C.byref(s), C.byref(h), C.byref(x), C.byref(P), C.byref(Q)))
    return dict(state_bytes=s.value, hist_bytes=h.value, scratch_bytes=x.value, P=P.value, Q=Q.value)


def pgc_init(cfg: pgc_config, d_state: int, d_hist: int, d_scratch: int, h_init_khat=None, stream: int = 0):
    out = _vp()
    init = None
    if h_init_khat is not None:
        init = np.ascontiguousarray(h_init_khat, dtype=np.float64)
    _check(lib().pgc_init(C.byref(cfg), _vp(d_state), _vp(d_hist), _vp(d_scratch), _ptr(init, _dp),
                          _vp(stream), C.byref(out)))
    return out.value


def pgc_step(ctx, n_steps: int, moments_every: int = 0):
    _check(lib().pgc_step(_vp(ctx), int(n_steps), int(moments_every)), _vp(ctx))


def pgc_moments(ctx, Q: int, capacity: int):
    T = C.c_int64()
    t = np.zeros(capacity)
    mean = np.zeros((capacity, 4))
    var = np.zeros((capacity, 4))
    nodes = np.zeros((capacity, Q, 4))
    _check(lib().pgc_moments(_vp(ctx), _ptr(t, _dp), _ptr(mean, _dp), _ptr(var, _dp), _ptr(nodes, _dp),
                             C.byref(T)), _vp(ctx))
    n = T.value
    return dict(t_fs=t[:n], mean=mean[:n], var=var[:n], nodes=nodes[:n])


def pgc_reconstruct_f(ctx, z, d: int, Nk: int):
    z = np.ascontiguousarray(np.asarray(z, dtype=np.float64).reshape(-1, max(d, 1)))
    nz = z.shape[0]
    H = np.zeros((nz, Nk, Nk), dtype=np.uint32)
    m = np.zeros(nz, dtype=np.uint32)
    _check(lib().pgc_reconstruct_f(_vp(ctx), _ptr(z, _dp), nz, _ptr(H, _u32p), _ptr(m, _u32p)), _vp(ctx))
    return H, m


def pgc_observe_at(ctx, z, d: int):
    """Observables [nz][4] = (V_x, V_y, energy, J_x) of the current state at the points z."""
    z = np.ascontiguousarray(np.asarray(z, dtype=np.float64).reshape(-1, max(d, 1)))
    out = np.zeros((z.shape[0], 4))
    _check(lib().pgc_observe_at(_vp(ctx), _ptr(z, _dp), z.shape[0], _ptr(out, _dp)), _vp(ctx))
    return out


def pgc_get_state(ctx, P: int, N: int):
    a = np.zeros((2, P, N))
    _check(lib().pgc_get_state(_vp(ctx), _ptr(a, _dp)), _vp(ctx))
    return a


def pgc_set_state(ctx, khat):
    a = np.ascontiguousarray(khat, dtype=np.float64)
    _check(lib().pgc_set_state(_vp(ctx), _ptr(a, _dp)), _vp(ctx))


def pgc_get_state_native(ctx, h_ptr: int):
    _check(lib().pgc_get_state_native(_vp(ctx), _vp(h_ptr)), _vp(ctx))


def pgc_set_state_native(ctx, h_ptr: int):
    _check(lib().pgc_set_state_native(_vp(ctx), _vp(h_ptr)), _vp(ctx))


def pgc_counters(ctx):
    a = np.zeros(8, dtype=np.uint64)
    _check(lib().pgc_counters(_vp(ctx), _ptr(a, _u64p)), _vp(ctx))
    return dict(zip(COUNTER_NAMES, [int(x) for x in a]))


def pgc_get_hist(ctx, Q: int, Nk: int):
    H = np.zeros((Q, Nk, Nk), dtype=np.uint32)
    m = np.zeros(Q, dtype=np.uint32)
    _check(lib().pgc_get_hist(_vp(ctx), _ptr(H, _u32p), _ptr(m, _u32p)), _vp(ctx))
    return H, m


def pgc_set_pipeline(ctx, on: bool):
    _check(lib().pgc_set_pipeline(_vp(ctx), 1 if on else 0), _vp(ctx))


def pgc_profile(ctx, every: int):
    _check(lib().pgc_profile(_vp(ctx), int(every)), _vp(ctx))


def pgc_profile_timeline(ctx, max_samples: int = 4096):
    """[n][4] ms: streaming-kernel start/end, collider-kernel start/end of each sampled step."""
    t = np.zeros((max_samples, 4))
    n = C.c_int64()
    _check(lib().pgc_profile_timeline(_vp(ctx), _ptr(t, _dp), int(max_samples), C.byref(n)), _vp(ctx))
    return t[: min(n.value, max_samples)]


def pgc_profile_read(ctx):
    a, b, n = C.c_double(), C.c_double(), C.c_int64()
    _check(lib().pgc_profile_read(_vp(ctx), C.byref(a), C.byref(b), C.byref(n)), _vp(ctx))
    return dict(phase1_ms=a.value, phase2_ms=b.value, samples=n.value)


def pgc_observe_static(ctx, d_hist_out: int, d_record_out: int, stream: int = 0):
    """No-allocation observation: histogram of the current state and one moment record, both
    written to caller-owned device buffers (see include/pgc.h)."""
    _check(lib().pgc_observe_static(_vp(ctx), _vp(d_hist_out), _vp(d_record_out), _vp(stream)), _vp(ctx))


def _check_batch(status, b=None):
    if status != PGC_OK:
        msg = lib().pgc_batch_last_error(b)
        raise PgcError(status, msg.decode() if msg else "")


def pgc_batch_query_sizes(ctxs):
    arr = (_vp * len(ctxs))(*ctxs)
    n = C.c_size_t()
    _check_batch(lib().pgc_batch_query_sizes(arr, len(ctxs), C.byref(n)))
    return n.value


def pgc_batch_create(ctxs, d_scratch: int, tile: int = 0):
    arr = (_vp * len(ctxs))(*ctxs)
    out = _vp()
    _check_batch(lib().pgc_batch_create(arr, len(ctxs), _vp(d_scratch), int(tile), C.byref(out)))
    return out.value


def pgc_batch_step(b, n_steps: int, moments_every: int = 0, use_graph: bool = True):
    _check_batch(lib().pgc_batch_step(_vp(b), int(n_steps), int(moments_every), int(bool(use_graph))), _vp(b))


def pgc_batch_autotune(b, steps_per_candidate: int):
    t = C.c_int32()
    ms = C.c_double()
    _check_batch(lib().pgc_batch_autotune(_vp(b), int(steps_per_candidate), C.byref(t), C.byref(ms)), _vp(b))
    return t.value, ms.value


def pgc_batch_launch_config(b):
    """(tile, threads per streaming block, particles per thread, streaming blocks per SM,
    collider blocks per SM) of a batch."""
    a = (C.c_int32 * 5)()
    _check_batch(lib().pgc_batch_launch_config(_vp(b), a), _vp(b))
    return dict(zip(["tile", "block", "ppt", "g1_per_sm", "g2_per_sm"], list(a)))


def pgc_batch_destroy(b):
    if b:
        lib().pgc_batch_destroy(_vp(b))


def pgc_adjoint_query_sizes(ctx, n_steps: int, ckpt_every: int) -> int:
    n = C.c_size_t()
    _check(lib().pgc_adjoint_query_sizes(_vp(ctx), int(n_steps), int(ckpt_every), C.byref(n)), _vp(ctx))
    return n.value


def pgc_adjoint(ctx, n_steps: int, ckpt_every: int, moments_every: int, window_steps: int, weights, d_work: int):
    """Returns (value[2] = (Jbar, Vbar), grad[4] = dL/d(E_lo, E_hi, eps0_lo, eps0_hi)) for
    L = weights[0] Jbar + weights[1] Vbar; see include/pgc.h."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    val = np.zeros(2)
    grad = np.zeros(4)
    _check(lib().pgc_adjoint(_vp(ctx), int(n_steps), int(ckpt_every), int(moments_every), int(window_steps),
                             _ptr(w, _dp), _vp(d_work), _ptr(val, _dp), _ptr(grad, _dp)), _vp(ctx))
    return val, grad


def pgc_destroy(ctx):
    if ctx:
        lib().pgc_destroy(_vp(ctx))


def pgc_launch_count() -> int:
    return int(lib().pgc_launch_count())


# ------------------------------------------------------------------------------------------
# configuration from a workload dictionary (paper_2404_19602_gb300.workloads)
# ------------------------------------------------------------------------------------------
def config_from(params: dict, max_outputs: int = 1024) -> pgc_config:
    c = pgc_config_default()
    p = params
    c.T_K = p.get("T_K", c.T_K)
    c.eps_F_eV = p.get("eps_F", c.eps_F_eV)
    c.eps0_eV.lo = p.get("eps0_lo", c.eps0_eV.lo)
    c.eps0_eV.hi = p.get("eps0_hi", c.eps0_eV.hi)
    c.Ex_Vcm.lo = p.get("Ex_lo", c.Ex_Vcm.lo)
    c.Ex_Vcm.hi = p.get("Ex_hi", c.Ex_Vcm.hi)
    c.mech_mask = p.get("mech_mask", c.mech_mask)
    c.alpha = p.get("alpha", c.alpha)
    c.Nk = p.get("Nk", c.Nk)
    c.Lk_hvF_eV = p.get("Lk_hvF", c.Lk_hvF_eV)
    c.degree_M = p.get("M", c.degree_M)
    c.quad_per_dim = p.get("Q1", c.quad_per_dim)
    c.n_particles = p.get("N", c.n_particles)
    c.dt_fs = p.get("dt_fs", c.dt_fs)
    c.seed = p.get("seed", c.seed)
    c.stream_id = p.get("stream_id", c.stream_id)
    prec = p.get("precision", "fp32")
    c.precision = PGC_FP64 if prec in ("fp64", 1) else PGC_FP32
    c.pauli_norm = p.get("pauli_norm", c.pauli_norm)
    c.final_state = p.get("final_state", c.final_state)
    c.n_theta_edge = p.get("n_theta", c.n_theta_edge)
    c.max_collisions = p.get("max_coll", c.max_collisions)
    c.max_outputs = max_outputs
    if (p.get("W_lo") or 0.0) > 0.0:   # width law: eps0(z) = hbar vF pi / W(z), W affine in z
        c.eps0_law = PGC_EPS0_WIDTH
        c.width_nm.lo = p["W_lo"]
        c.width_nm.hi = p.get("W_hi", p["W_lo"])
    c.splitting = p.get("splitting", c.splitting)   # PGC_SPLIT_LIE (0) or PGC_SPLIT_STRANG (1)
    c.tc_proj = p.get("tc_proj", c.tc_proj)         # PGC_TC_OFF (0), PGC_TC_F16X3 (1), PGC_TC_F16 (2)
    return c


class Simulation:
    """One ensemble on the current CUDA device; device buffers are torch tensors.

    >>> sim = Simulation(workloads.GAP_UQ_1E6)
    >>> sim.step(5000, moments_every=10)
    >>> m = sim.moments()       # t_fs, mean/var of (Vx, Vy, energy, Jx), per-node values
    """

    def __init__(self, params: dict, init_khat=None, max_outputs: int = 1024, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.params = dict(params)
        self.cfg = config_from(params, max_outputs)
        sz = pgc_query_sizes(self.cfg)
        self.P, self.Q = sz["P"], sz["Q"]
        self.N = int(self.cfg.n_particles)
        self.Nk = int(self.cfg.Nk)
        c = self.cfg
        eps_random = (c.width_nm.lo != c.width_nm.hi) if c.eps0_law == PGC_EPS0_WIDTH else (c.eps0_eV.lo != c.eps0_eV.hi)
        self.d = int(eps_random) + int(c.Ex_Vcm.lo != c.Ex_Vcm.hi)   # number of random inputs
        self.max_outputs = max_outputs
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        # Allocated with the context's stream current: torch's caching allocator then orders any
        # reuse of these blocks after the work queued on that stream (allocated under another
        # stream, a block freed there could be handed to this context while earlier work on it is
        # still pending).  The allocator returns 512-byte aligned blocks.
        with torch.cuda.stream(self.stream):
            self.state_buf = torch.empty(sz["state_bytes"], dtype=torch.uint8, device=dev)
            self.hist_buf = torch.empty(sz["hist_bytes"], dtype=torch.uint8, device=dev)
            self.scratch_buf = torch.empty(sz["scratch_bytes"], dtype=torch.uint8, device=dev)
        self.ctx = pgc_init(self.cfg, self.state_buf.data_ptr(), self.hist_buf.data_ptr(),
                            self.scratch_buf.data_ptr(), init_khat, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            pgc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_steps: int, moments_every: int = 0):
        pgc_step(self.ctx, n_steps, moments_every)

    def set_pipeline(self, on: bool):
        pgc_set_pipeline(self.ctx, on)

    def moments(self):
        return pgc_moments(self.ctx, self.Q, self.max_outputs)

    def state(self):
        return pgc_get_state(self.ctx, self.P, self.N)

    def set_state(self, khat):
        pgc_set_state(self.ctx, khat)

    def state_native(self):
        """The state in the device layout and precision, in a page-locked host tensor (uint8)."""
        import torch

        n = pgc_query_sizes(self.cfg)["state_bytes"]
        h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        pgc_get_state_native(self.ctx, h.data_ptr())
        return h

    def set_state_native(self, h):
        """Queue the upload of a state_native() tensor (the caller keeps it alive and unchanged
        until the context stream has passed the copy)."""
        n = pgc_query_sizes(self.cfg)["state_bytes"]
        if h.device.type != "cpu" or h.numel() * h.element_size() != n or not h.is_contiguous():
            raise ValueError("expected a contiguous host tensor of %d bytes" % n)
        pgc_set_state_native(self.ctx, h.data_ptr())

    def counters(self):
        return pgc_counters(self.ctx)

    def hist(self):
        return pgc_get_hist(self.ctx, self.Q, self.Nk)

    def reconstruct_f(self, z):
        return pgc_reconstruct_f(self.ctx, z, self.d, self.Nk)

    def observe_at(self, z):
        """(V_x, V_y, energy, J_x) at each point z (rows of shape [d], in [-1, 1]^d)."""
        return pgc_observe_at(self.ctx, z, self.d)


class BatchSimulation:
    """Many cases advanced together (pgc_batch_*).  Each case is a Simulation on one dedicated
    (non-default) stream, so that the step sequence can be captured into a CUDA graph."""

    def __init__(self, cases, max_outputs: int = 1024, tile: int = 0, stream=None):
        import torch

        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.sims = [Simulation(p, max_outputs=max_outputs, stream=self.stream) for p in cases]
        ctxs = [s.ctx for s in self.sims]
        n = pgc_batch_query_sizes(ctxs)
        with torch.cuda.stream(self.stream):   # allocated on the stream the batch runs on
            self.scratch_buf = torch.empty(max(n, 256), dtype=torch.uint8, device=self.sims[0].state_buf.device)
        self.batch = pgc_batch_create(ctxs, self.scratch_buf.data_ptr(), tile)

    def step(self, n_steps: int, moments_every: int = 0, use_graph: bool = True):
        pgc_batch_step(self.batch, n_steps, moments_every, use_graph)

    def autotune(self, steps_per_candidate: int = 3):
        return pgc_batch_autotune(self.batch, steps_per_candidate)

    def launch_config(self):
        return pgc_batch_launch_config(self.batch)

    def close(self):
        if getattr(self, "batch", None):
            pgc_batch_destroy(self.batch)
            self.batch = None
        for s in getattr(self, "sims", []):
            s.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def window_objective(params: dict, n_steps: int, moments_every: int, window_steps: int):
    """(Jbar, Vbar): averages over the moment records in (n_steps - window_steps, n_steps] of the
    mean and the variance over z of the current J_x, from a plain run (pgc_window_objective)."""
    sim = Simulation(params, max_outputs=n_steps // moments_every + 2)
    v = np.zeros(2)
    _check(lib().pgc_window_objective(_vp(sim.ctx), int(n_steps), int(moments_every), int(window_steps), _ptr(v, _dp)),
           _vp(sim.ctx))
    sim.close()
    return float(v[0]), float(v[1])


def adjoint(params: dict, n_steps: int, ckpt_every: int, moments_every: int, window_steps: int, weights=(1.0, 0.0)):
    """Pathwise gradient by the hand-written adjoint kernels (see pgc_adjoint in include/pgc.h)."""
    import torch

    sim = Simulation(params, max_outputs=n_steps // moments_every + 2)
    nbytes = pgc_adjoint_query_sizes(sim.ctx, n_steps, ckpt_every)
    with torch.cuda.stream(sim.stream):
        work = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=sim.state_buf.device)
    val, grad = pgc_adjoint(sim.ctx, n_steps, ckpt_every, moments_every, window_steps, weights, work.data_ptr())
    sim.close()
    return val, grad


def _torch_function():
    import torch

    class SteadyCurrent(torch.autograd.Function):
        """(Jbar, Vbar) of a run as a differentiable function of theta = (E_lo, E_hi, eps0_lo, eps0_hi)
        (V/cm, V/cm, eV, eV).  forward: a plain run; backward: the adjoint (events frozen, states
        checkpointed every ckpt_every steps and recomputed)."""

        @staticmethod
        def forward(fctx, theta, params, n_steps, moments_every, window_steps, ckpt_every):
            th = theta.detach().to("cpu", torch.float64).numpy()
            p = dict(params, Ex_lo=float(th[0]), Ex_hi=float(th[1]), eps0_lo=float(th[2]), eps0_hi=float(th[3]))
            fctx.cfg = (p, n_steps, moments_every, window_steps, ckpt_every)
            J, V = window_objective(p, n_steps, moments_every, window_steps)
            return torch.tensor([J, V], dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(fctx, grad_out):
            # one adjoint sweep for the weights (dLoss/dJbar, dLoss/dVbar)
            p, n_steps, every, window, ckpt = fctx.cfg
            g = grad_out.detach().to("cpu", torch.float64).numpy()
            _, grad = adjoint(p, n_steps, ckpt, every, window, weights=g)
            return torch.tensor(grad, dtype=torch.float64), None, None, None, None, None

    return SteadyCurrent


def steady_current(theta, params: dict, n_steps: int, moments_every: int, window_steps: int, ckpt_every: int = 250):
    """Differentiable (Jbar, Vbar); see SteadyCurrent."""
    return _torch_function().apply(theta, params, n_steps, moments_every, window_steps, ckpt_every)

