"""Thin ctypes binding of libg1g2 (include/g1g2.h): argument marshalling only.

Every step of the propagation runs in the CUDA library; nothing here computes
any part of the G1-G2 equations.  Host arrays are numpy (complex128, or
float64 for a real w); device arrays for `rhs` are torch CUDA tensors of
dtype complex128 (interleaved re/im doubles, the ABI layout).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libg1g2.so")

OK, EINVAL, ESYMM, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
SELFENERGY = {"HF": 0, "SOA": 1, "GW": 2, "GWX": 3, "TPP": 4, "TPH": 5, "DSL": 6}
PRECISION = {"fp64": 0, "tf32x3": 1, "bf16x4": 2}


class G1G2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("basis", ctypes.c_int), ("w_is_real", ctypes.c_int),
                ("sym_tol", ctypes.c_double), ("cuda_stream", ctypes.c_void_p), ("statistics", ctypes.c_int)]


class Obs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("n_particles", ctypes.c_double), ("e_one", ctypes.c_double),
                ("e_hf", ctypes.c_double), ("e_corr", ctypes.c_double), ("e_total", ctypes.c_double),
                ("pulse_work", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def load():
    """Load libg1g2.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libg1g2.so not found at {LIB_PATH}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    sig = {
        "g1g2_default_options": (None, [ctypes.POINTER(Options)]),
        "g1g2_init": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int,
                                     ctypes.POINTER(Options)]),
        "g1g2_init_factorised": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp,
                                                ctypes.c_int, ctypes.POINTER(Options)]),
        "g1g2_set_drive": (ctypes.c_int, [vp, _dp, ctypes.c_int, _dp, ctypes.c_int]),
        "g1g2_rhs": (ctypes.c_int, [vp, ctypes.c_double, vp, vp, vp, vp]),
        "g1g2_step": (ctypes.c_int, [vp, ctypes.c_double]),
        "g1g2_propagate": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Obs), _dp]),
        "g1g2_propagate_hfgkba": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int, _dp, ctypes.c_size_t]),
        "g1g2_observables": (ctypes.c_int, [vp, ctypes.POINTER(Obs), _dp, _dp]),
        "g1g2_get_state": (ctypes.c_int, [vp, _dp, _dp, _dp]),
        "g1g2_set_state": (ctypes.c_int, [vp, ctypes.c_double, _dp, _dp]),
        "g1g2_launch_count": (ctypes.c_longlong, [vp]),
        "g1g2_rhs_vjp": (ctypes.c_int, [vp, ctypes.c_double, vp, vp, vp, vp, vp, vp, vp]),
        "g1g2_adjoint": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                        _dp, _dp]),
        "g1g2_wait_selftest": (ctypes.c_int, [ctypes.c_int]),
        "g1g2_fp64_rate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
        "g1g2_g1_rhs_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int] + [vp] * 6),
        "g1g2_set_hubbard_path": (ctypes.c_int, [vp, ctypes.c_int]),
        "g1g2_hubbard_path": (ctypes.c_int, [vp]),
        "g1g2_set_adjoint_checkpoints": (ctypes.c_int, [vp, ctypes.c_int]),
        "g1g2_adjoint_plan": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "g1g2_profile": (ctypes.c_int, [vp, ctypes.c_int]),
        "g1g2_profile_report": (ctypes.c_int, [vp, ctypes.POINTER(KernelStat), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]),
        "g1g2_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "g1g2_last_error_detail": (ctypes.c_char_p, []),
        "g1g2_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check_noalloc_args(h, w, n, g2, dn, current_device):
    """Validate the tensors of g1_rhs_noalloc before anything is launched: contiguous
    complex128 CUDA tensors on the current device, h, n, dn of shape (nb, nb) and w, g2
    with nb^4 elements.  Returns nb; raises ValueError otherwise (a short
    or mistyped buffer would make the kernels read past its end)."""
    import torch
    if getattr(h, "dim", lambda: 0)() != 2 or h.shape[0] != h.shape[1]:
        raise ValueError("h must be an (nb, nb) tensor")
    nb = int(h.shape[0])
    for name, x, numel in (("h", h, nb * nb), ("w", w, nb ** 4), ("n", n, nb * nb), ("g2", g2, nb ** 4),
                           ("dn", dn, nb * nb)):
        if not getattr(x, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA tensor")
        if x.dtype != torch.complex128:
            raise ValueError(f"{name} must be complex128, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if x.numel() != numel or (numel == nb * nb and tuple(x.shape) != (nb, nb)):
            raise ValueError(f"{name} has shape {tuple(x.shape)}; nb = {nb} needs {numel} elements"
                             + (" as (nb, nb)" if numel == nb * nb else ""))
        if x.device.index != current_device:
            raise ValueError(f"{name} is on cuda:{x.device.index}, the current device is cuda:{current_device}")
    return nb


def g1_rhs_noalloc(h, w, n, g2, dn, restricted=False, stream=None):
    """G1 right-hand side dn = -i[hHF, n] - (I + I^dag) through g1g2_g1_rhs_noalloc, which
    allocates no device memory; all arguments are contiguous complex128 CUDA tensors on
    the current device (w and g2 with nb^4 elements, the ABI layout), dn is written.
    stream: a torch.cuda.Stream, a raw cudaStream_t handle (int), or None (default stream)."""
    import torch
    nb = check_noalloc_args(h, w, n, g2, dn, torch.cuda.current_device())
    if stream is None:
        handle = None
    elif isinstance(stream, torch.cuda.Stream):
        handle = stream.cuda_stream
    else:
        handle = int(stream)
    _check(load().g1g2_g1_rhs_noalloc(nb, 1 if restricted else 0, h.data_ptr(), w.data_ptr(), n.data_ptr(),
                                       g2.data_ptr(), dn.data_ptr(), handle))


def fp64_rate():
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s (g1g2_fp64_rate)."""
    v = ctypes.c_double()
    _check(load().g1g2_fp64_rate(ctypes.byref(v)))
    return v.value


def wait_selftest(limit_us=20000):
    """Return code of the bounded-wait self-test (ETIMEOUT is the expected result)."""
    return load().g1g2_wait_selftest(int(limit_us))


def _check(rc):
    if rc != OK:
        lib = load()
        raise G1G2Error(rc, f"{lib.g1g2_strerror(rc).decode()}: {lib.g1g2_last_error_detail().decode()}")


def _cptr(a):
    return a.ctypes.data_as(_dp)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


class Propagator:
    """One g1g2_ctx: state (G1 = n, G2), RK4 stepping, observables."""

    def __init__(self, h, w, n0, G2_0=None, selfenergy="SOA", precision="fp64", restricted=False,
                 sym_tol=1e-10, stream=None, bosons=False, factors=None):
        """w: the nb^4 interaction, or None with `factors` = L of shape (nfac, nb, nb), each L^P
        Hermitian or i times Hermitian, for the factorised w_ijkl = sum_P L^P_ik L^P_jl
        (g1g2_init_factorised)."""
        lib = load()
        self.nb = int(np.asarray(h).shape[0])
        self.restricted = restricted
        self.selfenergy = selfenergy
        opt = Options()
        lib.g1g2_default_options(ctypes.byref(opt))
        opt.precision = PRECISION[precision]
        opt.basis = 1 if restricted else 0
        opt.sym_tol = sym_tol
        opt.cuda_stream = stream
        opt.statistics = 1 if bosons else 0
        if (w is None) == (factors is None):
            raise ValueError("give exactly one of w and factors")
        x = np.asarray(w if factors is None else factors)
        if factors is not None and (x.ndim != 3 or x.shape[1:] != (self.nb, self.nb)):
            raise ValueError(f"factors must have shape (nfac, {self.nb}, {self.nb}), got {x.shape}")
        if np.isrealobj(x):
            wbuf = np.ascontiguousarray(x, dtype=np.float64)
            opt.w_is_real = 1
        else:
            wbuf = _c128(x)
        hb, nbuf = _c128(h), _c128(n0)
        gbuf = None if G2_0 is None else _c128(G2_0)
        gptr = None if gbuf is None else _cptr(gbuf)
        ctx = ctypes.c_void_p()
        if factors is None:
            rc = lib.g1g2_init(ctypes.byref(ctx), self.nb, _cptr(hb), _cptr(wbuf), _cptr(nbuf), gptr,
                               SELFENERGY[selfenergy], ctypes.byref(opt))
        else:
            rc = lib.g1g2_init_factorised(ctypes.byref(ctx), self.nb, _cptr(hb), _cptr(wbuf), int(x.shape[0]),
                                          _cptr(nbuf), gptr, SELFENERGY[selfenergy], ctypes.byref(opt))
        _check(rc)
        self._ctx = ctx
        self._lib = lib

    # -- lifecycle -------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.g1g2_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -----------------------------------------------------------
    def set_drive(self, D, drive):
        """h(t) = h + f(t) D; `drive` has .kind (1 gauss-sine, 2 piecewise linear) and .params."""
        if drive is None or D is None:
            _check(self._lib.g1g2_set_drive(self._ctx, None, 0, None, 0))
            return
        db = _c128(D)
        params = np.ascontiguousarray(drive.params, dtype=np.float64)
        _check(self._lib.g1g2_set_drive(self._ctx, _cptr(db), int(drive.kind), _cptr(params), len(params)))

    def rhs(self, t, n_dev, G2_dev, dn_dev, dG2_dev):
        """dn/dt and dG2/dt at (t, n, G2) into caller-owned device tensors (complex128, contiguous)."""
        for x in (n_dev, G2_dev, dn_dev, dG2_dev):
            if x is not None and not x.is_contiguous():
                raise ValueError("device tensors must be contiguous")
        ptr = lambda x: None if x is None else ctypes.c_void_p(x.data_ptr())
        _check(self._lib.g1g2_rhs(self._ctx, float(t), ptr(n_dev), ptr(G2_dev), ptr(dn_dev), ptr(dG2_dev)))

    def step(self, dt):
        _check(self._lib.g1g2_step(self._ctx, float(dt)))

    def propagate(self, dt, nsteps, obs_every=0):
        """Run nsteps RK4 steps; returns (list of observable dicts, density array) when obs_every > 0."""
        if obs_every <= 0:
            _check(self._lib.g1g2_propagate(self._ctx, float(dt), int(nsteps), 0, None, None))
            return [], None
        nrec = 1 + nsteps // obs_every
        obs = (Obs * nrec)()
        dens = np.zeros((nrec, self.nb))
        _check(self._lib.g1g2_propagate(self._ctx, float(dt), int(nsteps), int(obs_every), obs, _cptr(dens)))
        return [o.as_dict() for o in obs], dens

    def propagate_hfgkba(self, dt, nsteps, scratch_bytes=0):
        """Original memory-integral HF-GKBA (SOA, FP64 form) from the current uncorrelated
        state; returns n(t0 + m dt) for m = 0..nsteps as an (nsteps+1, nb, nb) array."""
        hist = np.zeros((int(nsteps) + 1, self.nb, self.nb), dtype=np.complex128)
        _check(self._lib.g1g2_propagate_hfgkba(self._ctx, float(dt), int(nsteps), _cptr(hist.view(np.float64)),
                                                int(scratch_bytes)))
        return hist

    def observables(self, double_occ=False):
        o = Obs()
        dens = np.zeros(self.nb)
        docc = np.zeros(self.nb // 2) if double_occ else None
        _check(self._lib.g1g2_observables(self._ctx, ctypes.byref(o), _cptr(dens),
                                          None if docc is None else _cptr(docc)))
        d = o.as_dict()
        d["density"] = dens
        if double_occ:
            d["double_occ"] = docc
        return d

    def get_state(self, with_g2=True):
        t = ctypes.c_double()
        n = np.zeros((self.nb, self.nb), dtype=np.complex128)
        g = np.zeros((self.nb,) * 4, dtype=np.complex128) if with_g2 else None
        _check(self._lib.g1g2_get_state(self._ctx, ctypes.byref(t), _cptr(n), None if g is None else _cptr(g)))
        return t.value, n, g

    def set_state(self, t, n, G2=None):
        nb_ = _c128(n)
        gb = None if G2 is None else _c128(G2)
        _check(self._lib.g1g2_set_state(self._ctx, float(t), _cptr(nb_), None if gb is None else _cptr(gb)))

    def rhs_vjp(self, t, n_dev, G2_dev, dn_bar, dG2_bar, n_bar, G2_bar, h_bar):
        """Cotangents of (n, G2, h^HF) from those of (dn/dt, dG2/dt) (device tensors, FP64 form)."""
        ptr = lambda x: ctypes.c_void_p(x.data_ptr())
        _check(self._lib.g1g2_rhs_vjp(self._ctx, float(t), ptr(n_dev), ptr(G2_dev), ptr(dn_bar), ptr(dG2_bar),
                                      ptr(n_bar), ptr(G2_bar), ptr(h_bar)))

    def adjoint(self, dt, nsteps, objective=0, ckpt_every=0, n_drive_params=0, grad_w=False):
        """Discrete adjoint from the current state: (J, grad_drive, grad_wscale, grad_h), and
        grad_w (nb^4 complex, on the symmetric interactions) as a fifth entry when asked.

        objective 0: mean double occupancy, 1: density imbalance, 2: energy absorbed.
        """
        J = ctypes.c_double()
        gd = np.zeros(max(n_drive_params, 1))
        gws = ctypes.c_double()
        gh = np.zeros((self.nb, self.nb), dtype=np.complex128)
        gw = np.zeros((self.nb,) * 4, dtype=np.complex128) if grad_w else None
        _check(self._lib.g1g2_adjoint(self._ctx, float(dt), int(nsteps), int(ckpt_every), int(objective),
                                      ctypes.byref(J), _cptr(gd) if n_drive_params else None, ctypes.byref(gws),
                                      _cptr(gh), None if gw is None else _cptr(gw)))
        out = (J.value, gd[:n_drive_params], gws.value, gh)
        return out + (gw,) if grad_w else out

    @property
    def hubbard_path(self):
        """True when the O(nb^4) Hubbard-basis right-hand side is in use."""
        return self._lib.g1g2_hubbard_path(self._ctx) == 1

    @hubbard_path.setter
    def hubbard_path(self, enable):
        _check(self._lib.g1g2_set_hubbard_path(self._ctx, 1 if enable else 0))

    CKPT = {"auto": 0, "device": 1, "host": 2}

    def set_adjoint_checkpoints(self, where="auto"):
        """Checkpoints of the adjoint in device memory, pinned host memory, or chosen by size ("auto")."""
        _check(self._lib.g1g2_set_adjoint_checkpoints(self._ctx, self.CKPT[where]))

    def adjoint_plan(self):
        """(interval, "device" | "host") of the last adjoint call."""
        k, w = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.g1g2_adjoint_plan(self._ctx, ctypes.byref(k), ctypes.byref(w)))
        return k.value, {0: None, 1: "device", 2: "host"}[w.value]

    def profile(self, enable=True):
        """Start (clearing old records) or stop per-kernel CUDA-event timing."""
        _check(self._lib.g1g2_profile(self._ctx, 1 if enable else 0))

    def profile_report(self):
        """{kernel name: (launches, total ms)} of the recorded launches (synchronises)."""
        stats = (KernelStat * 64)()
        n = ctypes.c_int()
        _check(self._lib.g1g2_profile_report(self._ctx, stats, 64, ctypes.byref(n)))
        return {stats[i].name.decode(): (stats[i].launches, stats[i].total_ms) for i in range(n.value)}

    @property
    def launch_count(self):
        return int(self._lib.g1g2_launch_count(self._ctx))


def save_checkpoint(prop, path):
    """Write the propagated state of `prop` (t, G1 = n, G2; the paper's initial-value data of
    Sec. III.F at time t) to `path` as a numpy .npz archive, with nb, the selfenergy and the
    basis for the check on resume.  The accumulated pulse work is an observable, not state:
    it restarts from zero after load_checkpoint (as after g1g2_set_state)."""
    t, n, g = prop.get_state()
    np.savez(path, t=np.float64(t), G1=n, G2=g, nb=np.int64(prop.nb), selfenergy=str(prop.selfenergy),
             restricted=bool(prop.restricted))


def load_checkpoint(prop, path):
    """Resume `prop` from a save_checkpoint archive (g1g2_set_state); returns t.  Refuses an
    archive of another nb, selfenergy or basis (ValueError).  Spin-restricted Hubbard GW keeps
    a same-spin block inside the context that set_state zeroes, so its resume is not exact."""
    with np.load(path) as z:
        for key, want in (("nb", prop.nb), ("selfenergy", str(prop.selfenergy)), ("restricted", bool(prop.restricted))):
            got = z[key].item()
            if got != want:
                raise ValueError(f"checkpoint has {key} = {got!r}, the propagator {want!r}")
        t, n, g = float(z["t"]), z["G1"], z["G2"]
    prop.set_state(t, n, g)
    return t


def from_workload(d, precision="fp64", stream=None):
    """Propagator for a workload dict of paper_2002_12717_gb300.inputs."""
    p = Propagator(d["h"], d["w"], d["n0"], d.get("G2_0"), selfenergy=d["selfenergy"], precision=precision,
                   restricted=d["restricted"], stream=stream)
    if d.get("D") is not None:
        p.set_drive(d["D"], d["drive"])
    return p
