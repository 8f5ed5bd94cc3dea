"""ctypes binding of libkn (include/kn.h): argument marshalling only.

Every step of the integration runs in the library's CUDA kernels.  Host
arrays are numpy; device arrays are torch CUDA tensors (torch supplies device
memory and the current stream, nothing else).  If libkn.so is missing or does
not load, every entry point raises KnError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass, fields

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkn.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "kn.h")

KN_OK, KN_ERR_INVALID_ARG, KN_ERR_CUDA, KN_ERR_NOMEM, KN_ERR_STATE, KN_ERR_INTERNAL = range(6)
ZONE_STATUS = {0: "ok", 1: "step_limit", 2: "dt_underflow", 3: "nonfinite", 4: "max_reject",
               5: "invalid", 6: "pending"}
PREC_FP64, PREC_MIXED, PREC_MIXED_FP64 = 0, 1, 2
METHOD_ASYMPTOTIC, METHOD_QSS = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1


class KnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libkn error {code}: {msg}")
        self.code = code


class _Desc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32), ("A", C.c_void_p),
                ("reac", C.c_void_p), ("prod", C.c_void_p), ("ln_k0", C.c_void_p),
                ("t9_exp", C.c_void_p)]


class _Zones(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")]


class _Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_reject", C.c_int32), ("kappa", C.c_double),
                ("eps_r", C.c_double), ("eps_c", C.c_double), ("y_min", C.c_double),
                ("grow_max", C.c_double), ("safety", C.c_double), ("shrink", C.c_double),
                ("dt_min_frac", C.c_double), ("max_steps", C.c_int64),
                ("threads_per_cta", C.c_int32), ("threads_per_zone", C.c_int32),
                ("use_graph", C.c_int32), ("lockstep", C.c_int32),
                ("replay_dt", C.c_void_p), ("replay_off", C.c_void_p), ("replay_len", C.c_void_p),
                ("mlp", C.c_void_p), ("record_features", C.c_void_p), ("record_labels", C.c_void_p),
                ("record_capacity", C.c_int64), ("record_count", C.c_void_p), ("mlp_margin", C.c_double),
                ("trace_features", C.c_void_p), ("trace_out", C.c_void_p), ("trace_dt", C.c_void_p),
                ("trace_capacity", C.c_int64), ("trace_count", C.c_void_p), ("follow_label", C.c_int32),
                ("method", C.c_int32), ("zone_ns", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("zones", C.c_int64), ("zones_ok", C.c_int64), ("steps", C.c_int64),
                ("rejects", C.c_int64), ("proposals_used", C.c_int64)]


class _Tiling(C.Structure):
    _fields_ = [("threads_per_cta", C.c_int32), ("threads_per_zone", C.c_int32),
                ("zone_steps_per_s", C.c_double), ("candidates", C.c_int32), ("pad", C.c_int32)]


_lib = None


def lib():
    """Load libkn.so (built by paper_1409_5826_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise KnError(-1, f"{LIB_PATH} is not built: run paper_1409_5826_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "kn_default_opts": (None, [C.POINTER(_Opts)]),
        "kn_last_error": (C.c_char_p, []),
        "kn_create_network": (I32, [C.POINTER(_Desc), C.POINTER(P)]),
        "kn_destroy_network": (I32, [P]),
        "kn_network_info": (I32, [P, P, P, P, P]),
        "kn_check_gather_tables": (I32, [C.POINTER(_Desc), I32, I32, P]),
        "kn_set_zone_conditions": (I32, [P, I32, C.POINTER(_Zones), I32, P]),
        "kn_integrate_batch": (I32, [P, I32, C.POINTER(_Opts), P]),
        "kn_get_abundances": (I32, [P, P, P, P, P, P, P, I32, P]),
        "kn_get_batch_stats": (I32, [P, I32, P, C.POINTER(_Stats)]),
        "kn_probe_step": (I32, [P, C.POINTER(_Opts), P, P, P, P, P, P]),
        "kn_integrate_noalloc": (I32, [P, I32, C.POINTER(_Zones), C.POINTER(_Opts), P, P, P, P, P, P, P]),
        "kn_autotune": (I32, [P, I32, C.POINTER(_Opts), I64, P, C.POINTER(_Tiling)]),
        "kn_advance_zones": (I32, [P, I32, P, P, P, I32, P]),
        "kn_set_binding_energies": (I32, [P, P]),
        "kn_get_energy": (I32, [P, P, I32, P]),
        "kn_measure_fp64_peak": (I32, [C.POINTER(C.c_double), P]),
        "kn_mlp_create": (I32, [C.POINTER(P)]),
        "kn_mlp_destroy": (I32, [P]),
        "kn_mlp_set_params": (I32, [P, P, P, P]),
        "kn_mlp_get_params": (I32, [P, P, P]),
        "kn_mlp_forward": (I32, [P, P, I32, P, P]),
        "kn_mlp_backward": (I32, [P, P, P, I32, P, P]),
        "kn_mlp_adam": (I32, [P, C.c_float, C.c_float, C.c_float, C.c_float, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_functions():
    """Names of every function declared in include/kn.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(kn_[a-z0-9_]+)\s*\(", txt)))


def _check(code):
    if code != KN_OK:
        raise KnError(code, lib().kn_last_error().decode())


def _stream_ptr(stream=None):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


@dataclass
class Opts:
    precision: int = PREC_MIXED
    max_reject: int = 60
    kappa: float = 1.0
    eps_r: float = 0.05
    eps_c: float = 1e-6
    y_min: float = 1e-10
    grow_max: float = 1.5
    safety: float = 0.9
    shrink: float = 0.5
    dt_min_frac: float = 1e-30
    max_steps: int = 10_000_000
    threads_per_cta: int = 0
    threads_per_zone: int = 0
    use_graph: int = 0
    lockstep: int = 0
    replay_dt: int = 0
    replay_off: int = 0
    replay_len: int = 0
    mlp: int = 0
    record_features: int = 0
    record_labels: int = 0
    record_capacity: int = 0
    record_count: int = 0
    mlp_margin: float = 0.5
    trace_features: int = 0
    trace_out: int = 0
    trace_dt: int = 0
    trace_capacity: int = 0
    trace_count: int = 0
    follow_label: int = 0
    method: int = METHOD_ASYMPTOTIC
    zone_ns: int = 0

    _PTRS = ("replay_dt", "replay_off", "replay_len", "mlp", "record_features", "record_labels", "record_count",
             "trace_features", "trace_out", "trace_dt", "trace_count", "zone_ns")

    def c(self) -> _Opts:
        o = _Opts()
        lib().kn_default_opts(C.byref(o))
        for f in fields(self):
            v = getattr(self, f.name)
            if f.name == "mlp" and v and not isinstance(v, int):
                v = v.h.value  # an MLP object
            setattr(o, f.name, (v or None) if f.name in self._PTRS else v)
        return o


def default_opts() -> _Opts:
    o = _Opts()
    lib().kn_default_opts(C.byref(o))
    return o


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def check_gather_tables(net, precision: int, threads_per_zone: int) -> dict:
    """Build and verify, on the host only, the gather tables the integrator
    would use for `net` (kn_check_gather_tables); returns their statistics."""
    keep = [_host(net.A, np.float64), _host(net.reac, np.int32), _host(net.prod, np.int32),
            _host(net.ln_k0, np.float64), _host(net.t9_exp, np.float64)]
    d = _Desc(int(net.n_species), int(net.n_reactions), *[a.ctypes.data for a in keep])
    st = np.zeros(4, np.int32)
    _check(lib().kn_check_gather_tables(C.byref(d), precision, threads_per_zone, st.ctypes.data))
    return {"piece_cap": int(st[0]), "slices": int(st[1]), "warp_terms_per_lane": int(st[2]),
            "table_bytes": int(st[3])}


class Network:
    """A network resident on the current device, plus its zones' state."""

    def __init__(self, net):
        self.N = int(net.n_species)
        self.R = int(net.n_reactions)
        self._keep = [_host(net.A, np.float64), _host(net.reac, np.int32), _host(net.prod, np.int32),
                      _host(net.ln_k0, np.float64), _host(net.t9_exp, np.float64)]
        d = _Desc(self.N, self.R, *[a.ctypes.data for a in self._keep])
        h = C.c_void_p()
        _check(lib().kn_create_network(C.byref(d), C.byref(h)))
        self.h = h
        self.Z = 0

    def info(self):
        v = [C.c_int32() for _ in range(4)]
        _check(lib().kn_network_info(self.h, *[C.byref(x) for x in v]))
        return dict(n_species=v[0].value, n_reactions=v[1].value, reactant_slots=v[2].value,
                    product_slots=v[3].value)

    def close(self):
        if getattr(self, "h", None):
            lib().kn_destroy_network(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_zones(self, zones, stream=None):
        """zones: kn_inputs.Zones (host numpy) or a dict of torch CUDA tensors
        with keys Y0, T0, rho0, tau, t_start, t_end, dt_trial."""
        names = ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")
        if isinstance(zones, dict):
            ts = [zones[n] for n in names]
            for t in ts:
                if not (t.is_cuda and t.is_contiguous()) or t.dtype.itemsize != 8:
                    raise ValueError("device zone arrays must be contiguous float64 CUDA tensors")
            Z = int(ts[1].shape[0])
            zc = _Zones(*[t.data_ptr() for t in ts])
            mem = MEM_DEVICE
            self._zkeep = ts
        else:
            arrs = [_host(getattr(zones, n), np.float64) for n in names]
            Z = int(arrs[1].shape[0])
            zc = _Zones(*[a.ctypes.data for a in arrs])
            mem = MEM_HOST
            self._zkeep = arrs
        _check(lib().kn_set_zone_conditions(self.h, Z, C.byref(zc), mem, C.c_void_p(_stream_ptr(stream))))
        self.Z = Z

    def get(self, stream=None):
        """Copy the results to host numpy arrays (synchronises the stream)."""
        Z, N = self.Z, self.N
        out = dict(Y=np.empty((Z, N)), t=np.empty(Z), dt_next=np.empty(Z),
                   steps=np.empty(Z, np.int64), rejects=np.empty(Z, np.int64),
                   status=np.empty(Z, np.int32))
        _check(lib().kn_get_abundances(self.h, *[out[k].ctypes.data for k in
                                                 ("Y", "t", "dt_next", "steps", "rejects", "status")],
                                       MEM_HOST, C.c_void_p(_stream_ptr(stream))))
        return out

    def get_device(self, out: dict, stream=None):
        """Copy the results into caller-owned torch CUDA tensors (keys as in get())."""
        keys = ("Y", "t", "dt_next", "steps", "rejects", "status")
        ptrs = [out[k].data_ptr() if k in out else None for k in keys]
        _check(lib().kn_get_abundances(self.h, *ptrs, MEM_DEVICE, C.c_void_p(_stream_ptr(stream))))
        return out

    def advance(self, T9, rho, t_end, stream=None):
        """Operator splitting: continue every zone into the next hydro interval at
        constant T9, rho (host arrays [Z]), carrying its last dt_next."""
        a = [_host(x, np.float64) for x in (T9, rho, t_end)]
        _check(lib().kn_advance_zones(self.h, self.Z, *[x.ctypes.data for x in a], MEM_HOST,
                                      C.c_void_p(_stream_ptr(stream))))

    def set_binding_energies(self, B):
        B = _host(B, np.float64)
        assert B.shape == (self.N,)
        _check(lib().kn_set_binding_energies(self.h, B.ctypes.data))

    def energy(self, stream=None) -> np.ndarray:
        E = np.empty(self.Z)
        _check(lib().kn_get_energy(self.h, E.ctypes.data, MEM_HOST, C.c_void_p(_stream_ptr(stream))))
        return E

    def probe(self, opts: Opts, stream=None):
        """One step from each zone's initial state (no accept test): F+, k, Y1, cons, rel."""
        import torch
        Z, N = self.Z, self.N
        dev = torch.device("cuda", torch.cuda.current_device())
        o = {k: torch.empty((Z, N) if k in ("Fp", "k", "Y1") else (Z,), dtype=torch.float64, device=dev)
             for k in ("Fp", "k", "Y1", "cons", "rel")}
        _check(lib().kn_probe_step(self.h, C.byref(opts.c()), *[o[k].data_ptr() for k in
                                                                ("Fp", "k", "Y1", "cons", "rel")],
                                   C.c_void_p(_stream_ptr(stream))))
        return {k: v.cpu().numpy() for k, v in o.items()}


def integrate_batch(nets, opts: Opts, stream=None):
    """Enqueue the integration of every zone of every network (asynchronous)."""
    arr = (C.c_void_p * len(nets))(*[n.h for n in nets])
    _check(lib().kn_integrate_batch(arr, len(nets), C.byref(opts.c()), C.c_void_p(_stream_ptr(stream))))


def batch_stats(nets, stream=None) -> dict:
    arr = (C.c_void_p * len(nets))(*[n.h for n in nets])
    s = _Stats()
    _check(lib().kn_get_batch_stats(arr, len(nets), C.c_void_p(_stream_ptr(stream)), C.byref(s)))
    return {f: getattr(s, f) for f, _ in _Stats._fields_}


MLP_FEATURES, MLP_HIDDEN, MLP_PARAMS = 64, 128, 24961


def mlp_pack(p: dict) -> np.ndarray:
    """Flat FP32 parameter array (W1, b1, W2, b2, w3, b3) from a dict of arrays."""
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def mlp_unpack(flat: np.ndarray) -> dict:
    F, H = MLP_FEATURES, MLP_HIDDEN
    o = 0
    out = {}
    for k, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, 1)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(shape)
        o += n
    return out


class MLP:
    """The learned-proposal network on the current device."""

    def __init__(self):
        h = C.c_void_p()
        _check(lib().kn_mlp_create(C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().kn_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: np.ndarray, mu, sigma):
        params = np.ascontiguousarray(params, np.float32)
        mu = np.ascontiguousarray(mu, np.float32)
        sigma = np.ascontiguousarray(sigma, np.float32)
        assert params.size == MLP_PARAMS and mu.size == MLP_FEATURES and sigma.size == MLP_FEATURES
        _check(lib().kn_mlp_set_params(self.h, params.ctypes.data, mu.ctypes.data, sigma.ctypes.data))

    def get_params(self):
        p = np.empty(MLP_PARAMS, np.float32)
        g = np.empty(MLP_PARAMS, np.float32)
        _check(lib().kn_mlp_get_params(self.h, p.ctypes.data, g.ctypes.data))
        return p, g

    def forward(self, feat, out, stream=None):
        """feat [B, 64] and out [B]: float32 CUDA tensors."""
        _check(lib().kn_mlp_forward(self.h, feat.data_ptr(), int(feat.shape[0]), out.data_ptr(),
                                    C.c_void_p(_stream_ptr(stream))))

    def backward(self, feat, labels, loss=None, stream=None):
        _check(lib().kn_mlp_backward(self.h, feat.data_ptr(), labels.data_ptr(), int(feat.shape[0]),
                                     loss.data_ptr() if loss is not None else None,
                                     C.c_void_p(_stream_ptr(stream))))

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(lib().kn_mlp_adam(self.h, lr, beta1, beta2, eps, C.c_void_p(_stream_ptr(stream))))


def autotune(nets, opts: Opts, max_steps: int = 400, stream=None) -> dict:
    """Time candidate tilings on the networks' current zones; the winner
    becomes their default tiling for this precision and form.  max_steps = 0
    times whole-batch trials (kn_autotune)."""
    arr = (C.c_void_p * len(nets))(*[n.h for n in nets])
    t = _Tiling()
    _check(lib().kn_autotune(arr, len(nets), C.byref(opts.c()), int(max_steps), C.c_void_p(_stream_ptr(stream)),
                             C.byref(t)))
    return {f: getattr(t, f) for f, _ in _Tiling._fields_ if f != "pad"}


def measure_fp64_peak(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    v = C.c_double()
    _check(lib().kn_measure_fp64_peak(C.byref(v), C.c_void_p(_stream_ptr(stream))))
    return v.value
