"""Thin ctypes binding of libbh.so (the C ABI in include/bh.h).

Argument marshalling only: every step of the path runs in the CUDA library.
torch is used for device memory (particle tensors) and for the current
stream.  There is no CPU fallback: ``load()`` raises when the library is
missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbh.so")

BH_OK, BH_E_INVAL, BH_E_NOMEM, BH_E_CUDA, BH_E_LIST_OVERFLOW, BH_E_TIMEOUT, BH_E_STATE = range(7)
BH_PREC_FP64, BH_PREC_FP32 = 0, 1
BH_FORCE_TREE_ONLY = 1
SYMBOLS = ("bh_create", "bh_batch_create", "bh_destroy", "bh_last_error", "bh_set_stream", "bh_build_tree", "bh_make_lists",
           "bh_compute_forces", "bh_step", "bh_step_host", "bh_sync", "bh_get_sizes", "bh_get_keys",
           "bh_get_root", "bh_get_tree", "bh_get_moments", "bh_get_groups", "bh_get_lists",
           "bh_get_counters", "bh_set_timing", "bh_get_timing", "bh_set_tuning", "bh_get_tuning", "bh_autotune",
           "bh_get_balance", "bh_get_diagnostics", "bh_sort_keys_static", "bh_split_f32",
           "bh_set_list_capacity", "bh_measure_peak", "bh_compute_potential")
BH_SCHED_GRID, BH_SCHED_STATIC, BH_SCHED_DYNAMIC = 0, 1, 2
BH_SORT_STATIC_MAX_N = 4194304
STAGES = ("keys", "sort", "permute", "tree", "moments", "groups", "lists", "split", "force", "contacts", "update",
          "refine")
BH_N_STAGES = len(STAGES)
BH_PEAK_FP32, BH_PEAK_FP64 = 0, 1


class bh_params(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("eps", ctypes.c_double), ("G", ctypes.c_double),
                ("M_central", ctypes.c_double), ("r_coll", ctypes.c_double), ("kappa", ctypes.c_double),
                ("eta", ctypes.c_double), ("dt", ctypes.c_double), ("n_g", ctypes.c_int),
                ("n_leaf", ctypes.c_int), ("order", ctypes.c_int), ("precision", ctypes.c_int),
                ("rebuild_every", ctypes.c_int), ("key_frame", ctypes.c_int),
                ("list_capacity", ctypes.c_int64), ("omega", ctypes.c_double)]


class bh_particles(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ("x", "y", "z", "vx", "vy", "vz", "m", "id", "ax", "ay", "az")] + [
        ("n", ctypes.c_int64)]


class bh_counters(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("n_groups", "n_pp", "n_pc", "n_evals", "n_rebuilds", "n_launches",
                                               "n_contacts", "n_pp_far", "n_one_walk_builds",
                                               "n_h2d_bytes", "n_d2h_bytes", "n_refined")] + [
        ("stage_ms", ctypes.c_double * BH_N_STAGES), ("stage_calls", ctypes.c_int64 * BH_N_STAGES),
        ("n_graph_builds", ctypes.c_int64), ("n_graph_build_redos", ctypes.c_int64),
        ("n_graph_captures", ctypes.c_int64)]


class bh_diagnostics(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
                ("angular_momentum", ctypes.c_double * 3), ("kinetic", ctypes.c_double),
                ("potential_central", ctypes.c_double), ("contact_candidates", ctypes.c_int64),
                ("contacts", ctypes.c_int64)]


class bh_tuning(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in ("n_g", "chunk", "warps", "sched", "order_by_cost", "graph", "order_window",
                                            "graph_contact_room", "graph_room")]


_lib = None


class BHError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libbh error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libbh.so (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA library must be built (no CPU fallback)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    vp = ctypes.POINTER(ctypes.c_void_p)
    lib.bh_create.argtypes = [ctypes.POINTER(bh_params), P, vp]
    lib.bh_batch_create.argtypes = [ctypes.POINTER(bh_params), ctypes.c_int, ctypes.POINTER(ctypes.c_int64), P, vp]
    lib.bh_destroy.argtypes = [P]
    lib.bh_last_error.argtypes = [P]
    lib.bh_last_error.restype = ctypes.c_char_p
    lib.bh_set_stream.argtypes = [P, P]
    lib.bh_build_tree.argtypes = [P, ctypes.POINTER(bh_particles)]
    lib.bh_make_lists.argtypes = [P]
    lib.bh_compute_forces.argtypes = [P, ctypes.POINTER(bh_particles), ctypes.c_int]
    lib.bh_step.argtypes = [P, ctypes.POINTER(bh_particles), ctypes.c_int]
    lib.bh_step_host.argtypes = [P, ctypes.POINTER(bh_particles), ctypes.c_int]
    lib.bh_sync.argtypes = [P]
    lib.bh_get_sizes.argtypes = [P] + [ctypes.POINTER(ctypes.c_int64)] * 5
    lib.bh_get_keys.argtypes = [P, P, P]
    lib.bh_get_root.argtypes = [P, P, P]
    lib.bh_get_tree.argtypes = [P] + [P] * 8
    lib.bh_get_moments.argtypes = [P, P, P, P]
    lib.bh_get_groups.argtypes = [P, P]
    lib.bh_get_lists.argtypes = [P, P, P, P, P]
    lib.bh_get_counters.argtypes = [P, ctypes.POINTER(bh_counters)]
    lib.bh_set_timing.argtypes = [P, ctypes.c_int]
    lib.bh_get_timing.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    lib.bh_set_tuning.argtypes = [P, ctypes.POINTER(bh_tuning)]
    lib.bh_get_tuning.argtypes = [P, ctypes.POINTER(bh_tuning)]
    lib.bh_autotune.argtypes = [P, ctypes.POINTER(bh_particles), ctypes.POINTER(ctypes.c_double)]
    lib.bh_get_balance.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.bh_get_diagnostics.argtypes = [P, ctypes.POINTER(bh_particles), ctypes.POINTER(bh_diagnostics)]
    lib.bh_sort_keys_static.argtypes = [P, P, P, P, ctypes.c_int64, P, ctypes.c_char_p, ctypes.c_size_t]
    lib.bh_split_f32.argtypes = [P, P, P, ctypes.c_int64, P]
    lib.bh_set_list_capacity.argtypes = [P, ctypes.c_int64]
    lib.bh_measure_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.bh_compute_potential.argtypes = [P, ctypes.POINTER(bh_particles), P, ctypes.POINTER(ctypes.c_double)]
    _lib = lib
    return lib


def _np(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(**kw) -> bh_params:
    p = bh_params()
    defaults = dict(theta=0.5, eps=0.0, G=1.0, M_central=0.0, r_coll=0.0, kappa=0.0, eta=0.0, dt=1e-3, n_g=64,
                    n_leaf=8, order=1, precision=BH_PREC_FP64, rebuild_every=4, key_frame=0, list_capacity=0,
                    omega=0.0)
    for k, v in {**defaults, **{k: v for k, v in kw.items() if k in defaults}}.items():
        setattr(p, k, v)
    return p


def _check_buffers(what: str, n: int, bufs):
    """Reject, before anything is launched, buffers the C side cannot check:
    bufs is a list of (name, tensor, torch dtype); each must have that dtype,
    exactly n elements, be contiguous and live on one CUDA device.  Returns
    that device."""
    import torch
    for name, t, dt in bufs:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{what}: {name} must be a torch tensor")
        if t.dtype != dt:
            raise ValueError(f"{what}: {name} must have dtype {dt}, not {t.dtype}")
        if t.numel() != n:
            raise ValueError(f"{what}: {name} has {t.numel()} elements, {n} expected")
        if not t.is_contiguous():
            raise ValueError(f"{what}: {name} must be contiguous")
    dev = bufs[0][1].device
    for name, t, _ in bufs:
        if not t.is_cuda:
            raise ValueError(f"{what}: {name} must be a CUDA tensor (got device {t.device})")
        if t.device != dev:
            raise ValueError(f"{what}: {name} is on {t.device}, {bufs[0][0]} on {dev}: all must share one device")
    return dev


def bh_sort_keys_static(keys, idx, keys_tmp, idx_tmp, stream=None):
    """Stable sort of the uint64 keys (device tensors, int64 dtype holding the
    bits) with idx (int32 dtype holding uint32) the input position of each
    sorted key; keys_tmp / idx_tmp are device scratch of the same sizes.
    All four tensors must be contiguous, on one CUDA device, with keys.numel()
    elements each.  The call runs with that device current, on the given
    stream (default: that device's current stream).  Nothing is allocated by
    the library; see bh.h for the limits."""
    import torch
    n = keys.numel() if isinstance(keys, torch.Tensor) else -1
    dev = _check_buffers("bh_sort_keys_static", n, [("keys", keys, torch.int64), ("idx", idx, torch.int32),
                                                     ("keys_tmp", keys_tmp, torch.int64),
                                                     ("idx_tmp", idx_tmp, torch.int32)])
    lib = load()
    with torch.cuda.device(dev):
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        buf = ctypes.create_string_buffer(256)
        rc = lib.bh_sort_keys_static(keys.data_ptr(), idx.data_ptr(), keys_tmp.data_ptr(), idx_tmp.data_ptr(), n,
                                     ctypes.c_void_p(stream), buf, len(buf))
    if rc != BH_OK:
        raise BHError(rc, buf.value.decode())
    return rc


def bh_split_f32(v, hi, lo, stream=None):
    """FP32 hi/lo split of the float64 device tensor v into the float32
    device tensors hi and lo (same length, contiguous, one CUDA device) on the
    given stream (default: that device's current stream), with that device
    current."""
    import torch
    n = v.numel() if isinstance(v, torch.Tensor) else -1
    dev = _check_buffers("bh_split_f32", n, [("v", v, torch.float64), ("hi", hi, torch.float32),
                                             ("lo", lo, torch.float32)])
    lib = load()
    with torch.cuda.device(dev):
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        rc = lib.bh_split_f32(v.data_ptr(), hi.data_ptr(), lo.data_ptr(), n, ctypes.c_void_p(stream))
    if rc != BH_OK:
        raise BHError(rc, "bh_split_f32 failed")
    return rc


def bh_measure_peak(kind: int) -> float:
    """Measured FMA peak of the current device in TFLOP/s (kind BH_PEAK_FP32
    or BH_PEAK_FP64)."""
    lib = load()
    v = ctypes.c_double()
    rc = lib.bh_measure_peak(int(kind), ctypes.byref(v))
    if rc != BH_OK:
        raise BHError(rc, "bh_measure_peak failed")
    return v.value


class Particles:
    """Caller-owned device arrays (torch tensors) in the layout bh.h expects."""
    FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "id", "ax", "ay", "az")

    def __init__(self, arrays: dict, device="cuda"):
        import torch
        n = len(arrays["x"])
        self.n = n
        self.t = {}
        for f in self.FIELDS:
            dt = torch.int64 if f == "id" else torch.float64
            if f in arrays:
                self.t[f] = torch.as_tensor(np.ascontiguousarray(arrays[f])).to(device=device, dtype=dt).contiguous()
            else:
                self.t[f] = torch.zeros(n, dtype=dt, device=device)
        self.struct = bh_particles(*(self.t[f].data_ptr() for f in self.FIELDS), n)

    def numpy(self) -> dict:
        return {f: self.t[f].cpu().numpy() for f in self.FIELDS}


class HostParticles:
    """Caller-owned HOST arrays for bh_step_host (page-locked when pinned)."""

    def __init__(self, arrays: dict, pinned: bool = False):
        n = len(arrays["x"])
        self.n = n
        self.a = {}
        self._keep = []
        for f in Particles.FIELDS:
            dt = np.int64 if f == "id" else np.float64
            if pinned:
                import torch
                t = torch.empty(n, dtype=torch.int64 if f == "id" else torch.float64, pin_memory=True)
                self._keep.append(t)
                v = t.numpy()
                v[:] = arrays[f] if f in arrays else 0
                self.a[f] = v
            else:
                self.a[f] = np.ascontiguousarray(arrays[f], dtype=dt).copy() if f in arrays else np.zeros(n, dt)
        self.struct = bh_particles(*(self.a[f].ctypes.data for f in Particles.FIELDS), n)


class Context:
    """Owns one bh_ctx; methods mirror the C entry points of the same names.
    offsets (patch particle offsets, n_patches + 1 entries) selects
    bh_batch_create."""

    def __init__(self, stream=None, offsets=None, **params):
        import torch
        self.lib = load()
        self.params = make_params(**params)
        h = ctypes.c_void_p()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.n_patches = 1
        if offsets is None:
            rc = self.lib.bh_create(ctypes.byref(self.params), ctypes.c_void_p(stream), ctypes.byref(h))
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            self.n_patches = len(off) - 1
            rc = self.lib.bh_batch_create(ctypes.byref(self.params), self.n_patches,
                                          off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          ctypes.c_void_p(stream), ctypes.byref(h))
        if rc != BH_OK:
            raise BHError(rc, "bh_create failed (see stderr)")
        self.h = h

    def _chk(self, rc):
        if rc != BH_OK:
            raise BHError(rc, self.lib.bh_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.bh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- entry points ----
    def bh_build_tree(self, P: Particles):
        return self._chk(self.lib.bh_build_tree(self.h, ctypes.byref(P.struct)))

    def bh_make_lists(self):
        return self._chk(self.lib.bh_make_lists(self.h))

    def bh_compute_forces(self, P: Particles, flags: int = 0):
        return self._chk(self.lib.bh_compute_forces(self.h, ctypes.byref(P.struct), flags))

    def bh_step(self, P: Particles, nsteps: int):
        return self._chk(self.lib.bh_step(self.h, ctypes.byref(P.struct), nsteps))

    def bh_step_host(self, H: HostParticles, nsteps: int):
        return self._chk(self.lib.bh_step_host(self.h, ctypes.byref(H.struct), nsteps))

    def bh_sync(self):
        return self._chk(self.lib.bh_sync(self.h))

    def bh_get_sizes(self):
        v = [ctypes.c_int64() for _ in range(5)]
        self._chk(self.lib.bh_get_sizes(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("n_nodes", "n_groups", "n_pp", "n_pc", "n_jj"), (x.value for x in v)))

    def bh_get_keys(self, n):
        k = np.empty(n, np.uint64)
        p = np.empty(n, np.uint32)
        self._chk(self.lib.bh_get_keys(self.h, _np(k), _np(p)))
        return k, p

    def bh_get_root(self):
        """(lo[3], L) for one patch; (lo[P, 3], L[P]) for a batch."""
        lo = np.empty((self.n_patches, 3))
        L = np.empty(self.n_patches)
        self._chk(self.lib.bh_get_root(self.h, _np(lo), _np(L)))
        if self.n_patches == 1:
            return lo[0], float(L[0])
        return lo, L

    def bh_get_tree(self):
        nn = self.bh_get_sizes()["n_nodes"]
        t = {"level": np.empty(nn, np.uint8), "begin": np.empty(nn, np.uint32), "end": np.empty(nn, np.uint32),
             "parent": np.empty(nn, np.int32), "first_child": np.empty(nn, np.int32),
             "nchild": np.empty(nn, np.uint8), "qlo": np.empty((nn, 3), np.uint32),
             "qhi": np.empty((nn, 3), np.uint32)}
        self._chk(self.lib.bh_get_tree(self.h, *[_np(t[f]) for f in ("level", "begin", "end", "parent",
                                                                        "first_child", "nchild", "qlo", "qhi")]))
        return t

    def bh_get_moments(self):
        nn = self.bh_get_sizes()["n_nodes"]
        M = np.empty(nn)
        c = np.empty((3, nn))
        Q = np.empty((nn, 6))
        self._chk(self.lib.bh_get_moments(self.h, _np(M), _np(c), _np(Q)))
        return {"M": M, "cx": c[0], "cy": c[1], "cz": c[2], "Q": Q}

    def bh_get_groups(self):
        ng = self.bh_get_sizes()["n_groups"]
        g = np.empty(max(ng, 1), np.int32)
        self._chk(self.lib.bh_get_groups(self.h, _np(g)))
        return g[:ng]

    def bh_get_lists(self):
        s = self.bh_get_sizes()
        ng = s["n_groups"]
        L = {"pp_off": np.empty(ng + 1, np.int64), "P": np.empty(max(s["n_pp"], 1), np.int32),
             "pc_off": np.empty(ng + 1, np.int64), "C": np.empty(max(s["n_pc"], 1), np.int32)}
        self._chk(self.lib.bh_get_lists(self.h, _np(L["pp_off"]), _np(L["P"]), _np(L["pc_off"]), _np(L["C"])))
        L["P"] = L["P"][: s["n_pp"]]
        L["C"] = L["C"][: s["n_pc"]]
        return L

    def bh_get_counters(self):
        """Counters; stage_ms / stage_calls are dicts keyed by stage name."""
        c = bh_counters()
        self._chk(self.lib.bh_get_counters(self.h, ctypes.byref(c)))
        out = {f: getattr(c, f) for f, _ in bh_counters._fields_ if not f.startswith("stage_")}
        out["stage_ms"] = dict(zip(STAGES, c.stage_ms[:]))
        out["stage_calls"] = dict(zip(STAGES, c.stage_calls[:]))
        return out

    def bh_set_list_capacity(self, entries: int):
        return self._chk(self.lib.bh_set_list_capacity(self.h, int(entries)))

    def bh_set_timing(self, enable: bool = True):
        return self._chk(self.lib.bh_set_timing(self.h, 1 if enable else 0))

    def bh_set_tuning(self, **kw):
        """Change some tuning fields (n_g, chunk, warps, sched, order_by_cost, graph)."""
        t = self.bh_get_tuning(as_struct=True)
        for k, v in kw.items():
            setattr(t, k, int(v))
        return self._chk(self.lib.bh_set_tuning(self.h, ctypes.byref(t)))

    def bh_get_tuning(self, as_struct: bool = False):
        t = bh_tuning()
        self._chk(self.lib.bh_get_tuning(self.h, ctypes.byref(t)))
        return t if as_struct else {f: getattr(t, f) for f, _ in bh_tuning._fields_}

    def bh_autotune(self, P: "Particles"):
        ms = ctypes.c_double()
        self._chk(self.lib.bh_autotune(self.h, ctypes.byref(P.struct), ctypes.byref(ms)))
        return ms.value

    def bh_get_diagnostics(self, P: "Particles"):
        d = bh_diagnostics()
        self._chk(self.lib.bh_get_diagnostics(self.h, ctypes.byref(P.struct), ctypes.byref(d)))
        return {"mass": d.mass, "momentum": np.array(d.momentum[:]), "angular_momentum": np.array(d.angular_momentum[:]),
                "kinetic": d.kinetic, "potential_central": d.potential_central,
                "contact_candidates": d.contact_candidates, "contacts": d.contacts}

    def bh_compute_potential(self, P: "Particles", phi=None):
        """Self-gravity potential energy W (and phi_i into the float64 device
        tensor phi of n elements when given)."""
        import torch
        ptr = None
        if phi is not None:
            if not (isinstance(phi, torch.Tensor) and phi.is_cuda and phi.dtype == torch.float64
                    and phi.is_contiguous() and phi.numel() == P.n):
                raise ValueError("phi must be a contiguous float64 CUDA tensor of n elements")
            ptr = phi.data_ptr()
        W = ctypes.c_double()
        self._chk(self.lib.bh_compute_potential(self.h, ctypes.byref(P.struct), ptr, ctypes.byref(W)))
        return W.value

    def bh_get_balance(self):
        b = ctypes.c_double()
        self._chk(self.lib.bh_get_balance(self.h, ctypes.byref(b)))
        return b.value

    def bh_get_timing(self, reset: bool = True):
        ms = ctypes.c_double()
        nl = ctypes.c_int64()
        self._chk(self.lib.bh_get_timing(self.h, ctypes.byref(ms), ctypes.byref(nl), 1 if reset else 0))
        return ms.value, nl.value
