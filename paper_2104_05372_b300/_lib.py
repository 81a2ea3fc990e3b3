"""ctypes binding of libgpa (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: it checks tensor dtypes / devices / contiguity, passes
raw device pointers and the current CUDA stream, allocates the workspace the
library's size query asks for (through torch, as plain device memory), and
raises ``GpaError`` on a nonzero status. There is no CPU fallback: if the
library or a CUDA device is missing, calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpa.so")

PREC_FP32, PREC_BF16_TC = 0, 1
SCATTER_AUTO, SCATTER_ATOMIC, SCATTER_WARPAGG, SCATTER_SORT = 0, 1, 2, 3
STRATEGIES = {"auto": 0, "atomic": 1, "warpagg": 2, "sort": 3, "smem": 4, "runs": 5}
ERR_ARG, ERR_INDEX, ERR_CUDA, ERR_WORKSPACE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_ALIGN = 1, 2, 3, 4, 5, 6, 7


class GpaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (code {code})")


_lock = threading.Lock()
_lib = None

_P = C.c_void_p
_I64, _I32, _D, _F, _SZ = C.c_int64, C.c_int32, C.c_double, C.c_float, C.c_size_t

_SIGS = {
    "gpa_status_string": ([_I32], C.c_char_p),
    "gpa_version": ([], _I32),
    "gpa_gmm_workspace_bytes": ([_I64, _I32, _I32, _I32, _I64], _SZ),
    "gmm_objective": ([_P] * 5 + [_I64, _I32, _I32, _D, _I32, _I32, _P, _P, _P, _P, _SZ, _P, _P], _I32),
    "gmm_vjp": ([_P] * 5 + [_I64, _I32, _I32, _D, _I32, _I32, _P, _P, _D, _P, _P, _P, _P, _P, _P, _SZ, _P, _P],
                _I32),
    "gpa_gmm_jvp_workspace_bytes": ([_I64, _I32, _I32], _SZ),
    "gmm_jvp": ([_P] * 5 + [_I64, _I32, _I32, _D, _I32] + [_P] * 4 + [_P, _P, _P, _P, _SZ, _P, _P], _I32),
    "gpa_gmm_exchange_len": ([_I32, _I32], _I64),
    "gmm_vjp_partial": ([_P] * 5 + [_I64, _I32, _I32, _D, _I32, _I32, _P, _P, _D, _P, _P, _SZ, _P, _P], _I32),
    "gmm_vjp_finalize": ([_P] * 4 + [_I64, _I32, _I32, _D, _I32, _I32, _D, _P, _P, _P, _P, _P, _P, _P, _SZ, _P,
                                     _P], _I32),
    "gpa_reproj_workspace_bytes": ([_I32, _I32, _I64], _SZ),
    "reproj_residual": ([_P, _P, _P, _P, _I32, _I32, _I64, _P, _P, _SZ, _P, _P], _I32),
    "reproj_vjp": ([_P, _P, _P, _P, _I32, _I32, _I64, _P, _P, _I32, _P, _I32, _P, _SZ, _P, _P], _I32),
    "reproj_residual_vjp": ([_P, _P, _P, _P, _I32, _I32, _I64, _F, _P, _P, _P, _I32, _P, _I32, _P, _SZ, _P, _P],
                            _I32),
    "reproj_jvp": ([_P, _P, _P, _P, _P, _I32, _I32, _I64, _P, _P, _SZ, _P, _P], _I32),
    "reproj_residual_sorted": ([_P, _P, _P, _P, _I32, _I32, _I64, _P, _P, _I32, _P, _SZ, _P, _P], _I32),
    "gpa_reproj_gn_workspace_bytes": ([_I32, _I32, _I64], _SZ),
    "reproj_normal_eqs": ([_P] * 4 + [_I32, _I32, _I64] + [_P] * 3 + [_I32, _I32] + [_P] * 3 + [_I32, _P, _P, _SZ, _P, _P],
                          _I32),
    "reproj_vjp_noalloc": ([_P, _P, _P, _P, _I32, _I32, _I64, _P, _P, _I32, _P, _P, _P], _I32),
    "gpa_plan_bytes": ([_I64, _I32], _SZ),
    "gpa_plan_workspace_bytes": ([_I64, _I32], _SZ),
    "gpa_obs_plan_build": ([_P, _I64, _I32, _I32, _P, _SZ, _P, _SZ, _P, _P], _I32),
    "gpa_index_plan_build": ([_P, _I64, _I32, _P, _SZ, _P, _SZ, _P, _P], _I32),
    "accum_scatter_add": ([_P, _P, _I64, _I32, _I32, _P, _I32, _I32, _P, _P, _P], _I32),
    "gpa_gmm_batched_workspace_bytes": ([_P, _I32, _I64], _SZ),
    "gmm_batched_prepare": ([_P, _I32, _I64, _P, _SZ, _P], _I32),
    "gmm_batched_vjp": ([_P, _I32, _I64, _I32, _P, _SZ, _P, _P], _I32),
    "gpa_gmm_batched_workspace_bytes_opts": ([_P, _I32, _P], _SZ),
    "gpa_gmm_vjp_host_workspace_bytes": ([_I64, _I32, _I32, _I32, _I64], _SZ),
    "gmm_vjp_host": ([_P] * 5 + [_I64, _I32, _I32, _D, _I32, _I32, _D] + [_P] * 5 + [_I64, _P, _SZ, _P, _P], _I32),
    "gmm_batched_prepare_opts": ([_P, _I32, _P, _P, _SZ, _P], _I32),
    "gmm_batched_vjp_opts": ([_P, _I32, _P, _P, _SZ, _P, _P], _I32),
    "gpa_check_bounded_wait": ([_I64, _P, _P, _P], _I32),
    "gpa_trace_enable": ([_I32], None),
    "gpa_trace_summary": ([C.c_char_p, _SZ], _I32),
}


def load():
    """Load libgpa.so (built in-tree by ``paper_2104_05372_b300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libgpa.so not found at {LIB_PATH}; run "
                                   "`python -m paper_2104_05372_b300.build` first")
            lib = C.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def gpa_trace_enable(on: bool = True):
    load().gpa_trace_enable(1 if on else 0)


def gpa_trace_summary():
    """{kernel name: (launches, total_ms)} since the last summary."""
    lib = load()
    need = lib.gpa_trace_summary(None, 0)
    buf = C.create_string_buffer(need + 1)
    lib.gpa_trace_summary(buf, need + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def exported_symbols():
    return list(_SIGS)


def status_string(code: int) -> str:
    return load().gpa_status_string(int(code)).decode()


def version() -> int:
    return int(load().gpa_version())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ok(code, where):
    if code != 0:
        raise GpaError(int(code), where)


def workspace(nbytes: int, device) -> torch.Tensor:
    """Device scratch buffer of at least nbytes (256-byte aligned by the allocator)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------------------
# GMM
# ---------------------------------------------------------------------------
def gpa_gmm_workspace_bytes(n, d, k, prec=PREC_FP32, logjoint_points=0) -> int:
    return int(load().gpa_gmm_workspace_bytes(int(n), int(d), int(k), int(prec), int(logjoint_points)))


def _gmm_params(x, alpha, mu, q, l):
    _check(x, torch.float32, "x")
    n, d = x.shape
    k = alpha.shape[0]
    t = d * (d - 1) // 2
    _check(alpha, torch.float32, "alpha", (k,))
    _check(mu, torch.float32, "mu", (k, d))
    _check(q, torch.float32, "q", (k, d))
    _check(l, torch.float32, "l", (k, t))
    return n, d, k


def gmm_objective(x, alpha, mu, q, l, gamma=1.0, m=0, prec=PREC_FP32, out=None, lse_out=None,
                  logjoint_out=None, ws=None, status=None, stream=None):
    """Objective f into ``out`` (device float64 [1]); returns ``out``."""
    n, d, k = _gmm_params(x, alpha, mu, q, l)
    dev = x.device
    out = torch.empty(1, dtype=torch.float64, device=dev) if out is None else _check(out, torch.float64, "out")
    if lse_out is not None:
        _check(lse_out, torch.float32, "lse_out", (n,))
    if logjoint_out is not None:
        _check(logjoint_out, torch.float32, "logjoint_out", (k, n))
    nb = gpa_gmm_workspace_bytes(n, d, k, prec, 128)
    if ws is None:
        ws = workspace(nb, dev)
    rc = load().gmm_objective(_ptr(x), _ptr(alpha), _ptr(mu), _ptr(q), _ptr(l), n, d, k, float(gamma), int(m),
                              int(prec), _ptr(out), _ptr(lse_out), _ptr(logjoint_out), _ptr(ws), ws.numel(),
                              _ptr(status), _stream(stream))
    _ok(rc, "gmm_objective")
    return out


def gmm_vjp(x, alpha, mu, q, l, gamma=1.0, m=0, prec=PREC_FP32, logjoint_in=None, lse_in=None, seed=1.0,
            d_alpha=None, d_mu=None, d_q=None, d_l=None, out=None, ws=None, logjoint_points=0, status=None,
            stream=None):
    """seed * grad f added into (d_alpha, d_mu, d_q, d_l) (zeros if not given); returns them."""
    n, d, k = _gmm_params(x, alpha, mu, q, l)
    dev = x.device
    t = d * (d - 1) // 2
    d_alpha = torch.zeros(k, dtype=torch.float32, device=dev) if d_alpha is None else d_alpha
    d_mu = torch.zeros(k, d, dtype=torch.float32, device=dev) if d_mu is None else d_mu
    d_q = torch.zeros(k, d, dtype=torch.float32, device=dev) if d_q is None else d_q
    d_l = torch.zeros(k, t, dtype=torch.float32, device=dev) if d_l is None else d_l
    _check(d_alpha, torch.float32, "d_alpha", (k,))
    _check(d_mu, torch.float32, "d_mu", (k, d))
    _check(d_q, torch.float32, "d_q", (k, d))
    _check(d_l, torch.float32, "d_l", (k, t))
    if logjoint_in is not None:
        _check(logjoint_in, torch.float32, "logjoint_in", (k, n))
    if lse_in is not None:
        _check(lse_in, torch.float32, "lse_in", (n,))
    if out is not None:
        _check(out, torch.float64, "out")
    if ws is None:
        lp = 128 if logjoint_in is not None else logjoint_points
        ws = workspace(gpa_gmm_workspace_bytes(n, d, k, prec, lp), dev)
    rc = load().gmm_vjp(_ptr(x), _ptr(alpha), _ptr(mu), _ptr(q), _ptr(l), n, d, k, float(gamma), int(m), int(prec),
                        _ptr(logjoint_in), _ptr(lse_in), float(seed), _ptr(d_alpha), _ptr(d_mu), _ptr(d_q),
                        _ptr(d_l), _ptr(out), _ptr(ws), ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "gmm_vjp")
    return d_alpha, d_mu, d_q, d_l


def gmm_jvp(x, alpha, mu, q, l, v_alpha, v_mu, v_q, v_l, gamma=1.0, m=0, df_out=None, f_out=None,
            lse_dot_out=None, ws=None, status=None, stream=None):
    """Directional derivative df[v] into ``df_out`` (device float64 [1]); returns it."""
    n, d, k = _gmm_params(x, alpha, mu, q, l)
    t = d * (d - 1) // 2
    dev = x.device
    _check(v_alpha, torch.float32, "v_alpha", (k,))
    _check(v_mu, torch.float32, "v_mu", (k, d))
    _check(v_q, torch.float32, "v_q", (k, d))
    _check(v_l, torch.float32, "v_l", (k, t))
    df_out = torch.empty(1, dtype=torch.float64, device=dev) if df_out is None else _check(df_out, torch.float64,
                                                                                          "df_out")
    if f_out is not None:
        _check(f_out, torch.float64, "f_out")
    if lse_dot_out is not None:
        _check(lse_dot_out, torch.float32, "lse_dot_out", (n,))
    if ws is None:
        ws = workspace(int(load().gpa_gmm_jvp_workspace_bytes(n, d, k)), dev)
    rc = load().gmm_jvp(_ptr(x), _ptr(alpha), _ptr(mu), _ptr(q), _ptr(l), n, d, k, float(gamma), int(m),
                        _ptr(v_alpha), _ptr(v_mu), _ptr(v_q), _ptr(v_l), _ptr(df_out), _ptr(f_out),
                        _ptr(lse_dot_out), _ptr(ws), ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "gmm_jvp")
    return df_out


def gpa_gmm_exchange_len(d, k) -> int:
    return int(load().gpa_gmm_exchange_len(int(d), int(k)))


def gmm_vjp_partial(x, alpha, mu, q, l, gamma=1.0, m=0, prec=PREC_FP32, logjoint_in=None, lse_in=None,
                    seed=1.0, exch=None, ws=None, logjoint_points=0, status=None, stream=None):
    """Exchange vector (device float64) of this shard of points added (+=) into
    ``exch`` (zeros if not given); returns it."""
    n, d, k = _gmm_params(x, alpha, mu, q, l)
    dev = x.device
    e = gpa_gmm_exchange_len(d, k)
    exch = torch.zeros(e, dtype=torch.float64, device=dev) if exch is None else _check(exch, torch.float64,
                                                                                        "exch", (e,))
    if logjoint_in is not None:
        _check(logjoint_in, torch.float32, "logjoint_in", (k, n))
    if lse_in is not None:
        _check(lse_in, torch.float32, "lse_in", (n,))
    if ws is None:
        lp = 128 if logjoint_in is not None else logjoint_points
        ws = workspace(gpa_gmm_workspace_bytes(n, d, k, prec, lp), dev)
    rc = load().gmm_vjp_partial(_ptr(x), _ptr(alpha), _ptr(mu), _ptr(q), _ptr(l), n, d, k, float(gamma), int(m),
                                int(prec), _ptr(logjoint_in), _ptr(lse_in), float(seed), _ptr(exch), _ptr(ws),
                                ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "gmm_vjp_partial")
    return exch


def _check_host(t, name, shape):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.is_cuda:
        raise ValueError(f"{name} must be in host memory")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be torch.float32, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def gpa_gmm_vjp_host_workspace_bytes(n, d, k, prec=PREC_FP32, chunk_points=0) -> int:
    return int(load().gpa_gmm_vjp_host_workspace_bytes(int(n), int(d), int(k), int(prec), int(chunk_points)))


def gmm_vjp_host(x, alpha, mu, q, l, gamma=1.0, m=0, prec=PREC_FP32, seed=1.0, chunk_points=0, d_alpha=None,
                 d_mu=None, d_q=None, d_l=None, out=None, ws=None, device=None, status=None, stream=None):
    """gmm_vjp_host: points and parameters in host memory (pinned for
    asynchronous copies), seed * grad f and the objective WRITTEN to host
    tensors (pinned ones allocated if not given). The results are complete once
    ``stream`` (default: the current stream of ``device``) has run the call;
    returns (d_alpha, d_mu, d_q, d_l, out)."""
    n, d = x.shape
    k = alpha.shape[0]
    t = d * (d - 1) // 2
    for v, name, shape in ((x, "x", (n, d)), (alpha, "alpha", (k,)), (mu, "mu", (k, d)), (q, "q", (k, d)),
                           (l, "l", (k, t))):
        _check_host(v, name, shape)

    def host_out(v, name, shape):
        return torch.empty(shape, dtype=torch.float32).pin_memory() if v is None else _check_host(v, name, shape)
    d_alpha = host_out(d_alpha, "d_alpha", (k,))
    d_mu = host_out(d_mu, "d_mu", (k, d))
    d_q = host_out(d_q, "d_q", (k, d))
    d_l = host_out(d_l, "d_l", (k, t))
    out = torch.empty(1, dtype=torch.float64).pin_memory() if out is None else out
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if ws is None:
        nb = gpa_gmm_vjp_host_workspace_bytes(n, d, k, prec, chunk_points)
        if nb == 0:
            raise GpaError(ERR_ARG, "gpa_gmm_vjp_host_workspace_bytes")
        ws = workspace(nb, dev)
    s = torch.cuda.current_stream(dev) if stream is None else stream
    rc = load().gmm_vjp_host(_hptr(x), _hptr(alpha), _hptr(mu), _hptr(q), _hptr(l), n, d, k, float(gamma), int(m),
                             int(prec), float(seed), _hptr(d_alpha), _hptr(d_mu), _hptr(d_q), _hptr(d_l), _hptr(out),
                             int(chunk_points), _ptr(ws), ws.numel(), _ptr(status), C.c_void_p(s.cuda_stream))
    _ok(rc, "gmm_vjp_host")
    return d_alpha, d_mu, d_q, d_l, out


def _hptr(t):
    """Host address of a CPU tensor's data (None for an empty tensor)."""
    return C.c_void_p(t.data_ptr()) if t.numel() else None


def gmm_vjp_finalize(alpha, mu, q, l, n_total, exch, gamma=1.0, m=0, prec=PREC_FP32, seed=1.0, d_alpha=None,
                     d_mu=None, d_q=None, d_l=None, out=None, ws=None, status=None, stream=None):
    """seed * grad f over all shards added into (d_alpha, d_mu, d_q, d_l) from
    the summed exchange vector; returns them."""
    k, d = mu.shape
    t = d * (d - 1) // 2
    dev = mu.device
    _check(alpha, torch.float32, "alpha", (k,))
    _check(mu, torch.float32, "mu", (k, d))
    _check(q, torch.float32, "q", (k, d))
    _check(l, torch.float32, "l", (k, t))
    _check(exch, torch.float64, "exch", (gpa_gmm_exchange_len(d, k),))
    d_alpha = torch.zeros(k, dtype=torch.float32, device=dev) if d_alpha is None else d_alpha
    d_mu = torch.zeros(k, d, dtype=torch.float32, device=dev) if d_mu is None else d_mu
    d_q = torch.zeros(k, d, dtype=torch.float32, device=dev) if d_q is None else d_q
    d_l = torch.zeros(k, t, dtype=torch.float32, device=dev) if d_l is None else d_l
    _check(d_alpha, torch.float32, "d_alpha", (k,))
    _check(d_mu, torch.float32, "d_mu", (k, d))
    _check(d_q, torch.float32, "d_q", (k, d))
    _check(d_l, torch.float32, "d_l", (k, t))
    if out is not None:
        _check(out, torch.float64, "out")
    if ws is None:
        ws = workspace(gpa_gmm_workspace_bytes(1, d, k, prec, 128), dev)
    rc = load().gmm_vjp_finalize(_ptr(alpha), _ptr(mu), _ptr(q), _ptr(l), int(n_total), d, k, float(gamma), int(m),
                                 int(prec), float(seed), _ptr(exch), _ptr(d_alpha), _ptr(d_mu), _ptr(d_q),
                                 _ptr(d_l), _ptr(out), _ptr(ws), ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "gmm_vjp_finalize")
    return d_alpha, d_mu, d_q, d_l


class GmmInstance(C.Structure):
    """C layout of gpa_gmm_instance (include/gpa.h)."""
    _fields_ = [("x", C.c_void_p), ("alpha", C.c_void_p), ("mu", C.c_void_p), ("q", C.c_void_p),
                ("l", C.c_void_p), ("d_alpha", C.c_void_p), ("d_mu", C.c_void_p), ("d_q", C.c_void_p),
                ("d_l", C.c_void_p), ("out", C.c_void_p), ("n", C.c_int64), ("d", C.c_int32), ("k", C.c_int32),
                ("gamma", C.c_double), ("m", C.c_int32), ("seed", C.c_double), ("prec", C.c_int32)]


BATCH_CLASSES = 5  # padded dimension 8, 16, 32, 64, 128 (GPA_BATCH_CLASSES)
BATCH_CLASS_DP = (8, 16, 32, 64, 128)


def batch_class(d: int, prec: int = 0) -> int:
    """Class index of an instance of dimension d in the batched form (the
    tensor-core instances by their padded dimension 64 / 128)."""
    if prec == PREC_BF16_TC:
        return 3 if d <= 64 else 4
    return 0 if d <= 8 else 1 if d <= 16 else 2 if d <= 32 else 3 if d <= 64 else 4


class BatchedOpts(C.Structure):
    """C layout of gpa_batched_opts (include/gpa.h): per class chunk_points,
    ctas_per_sm, small_groups."""
    _fields_ = [("chunk_points", C.c_int64 * BATCH_CLASSES), ("ctas_per_sm", C.c_int32 * BATCH_CLASSES),
                ("small_groups", C.c_int32 * BATCH_CLASSES)]

    @classmethod
    def make(cls, per_class):
        """per_class: {class index: {"chunk_points", "ctas_per_sm", "small_groups"}}; classes not
        given take (4096, 0, 0)."""
        o = cls()
        for c in range(BATCH_CLASSES):
            v = per_class.get(c, per_class.get(str(c), {}))
            o.chunk_points[c] = int(v.get("chunk_points", 4096))
            o.ctas_per_sm[c] = int(v.get("ctas_per_sm", 0))
            o.small_groups[c] = int(v.get("small_groups", 0))
        return o


class GmmBatch:
    """Device tensors and descriptors of a batch of GMM instances.

    instances: list of dicts with keys x, alpha, mu, q, l (device float32
    tensors) and optionally gamma, m, seed, prec (PREC_FP32 or PREC_BF16_TC).
    Gradient buffers (zeros) and a float64 objective per instance are
    allocated here.
    """

    def __init__(self, instances, chunk_points=4096, opts=None):
        """opts: None (every class at chunk_points, CTAs per SM as given to
        run) or {class index: {"chunk_points", "ctas_per_sm", "small_groups"}}
        (the _opts entry points; run's ctas_per_sm is then ignored)."""
        self.chunk_points = int(chunk_points)
        self.opts = None if opts is None else BatchedOpts.make(opts)
        dev = instances[0]["x"].device
        shapes = [_gmm_params(i["x"], i["alpha"], i["mu"], i["q"], i["l"]) for i in instances]
        # every gradient and objective of the batch in one buffer: one memset clears them
        sizes = [k + 2 * k * d + k * (d * (d - 1) // 2) for n, d, k in shapes]
        self.flat = torch.zeros(sum(sizes), dtype=torch.float32, device=dev)
        self.outs = torch.zeros(len(instances), dtype=torch.float64, device=dev)
        self.tensors = []
        arr = (GmmInstance * len(instances))()
        off = 0
        for i, (inst, (n, d, k)) in enumerate(zip(instances, shapes)):
            t = d * (d - 1) // 2
            parts = []
            for numel, shape in ((k, (k,)), (k * d, (k, d)), (k * d, (k, d)), (k * t, (k, t))):
                parts.append(self.flat[off:off + numel].view(shape))
                off += numel
            out = self.outs[i:i + 1]
            self.tensors.append((inst, parts, out))
            arr[i] = GmmInstance(inst["x"].data_ptr(), inst["alpha"].data_ptr(), inst["mu"].data_ptr(),
                                 inst["q"].data_ptr(), inst["l"].data_ptr() if t > 0 else 0,
                                 parts[0].data_ptr(), parts[1].data_ptr(), parts[2].data_ptr(),
                                 parts[3].data_ptr() if t > 0 else 0, out.data_ptr(), n, d, k,
                                 float(inst.get("gamma", 1.0)), int(inst.get("m", 0)), float(inst.get("seed", 1.0)),
                                 int(inst.get("prec", PREC_FP32)))
        self.desc = arr
        self.n_inst = len(instances)
        self.pairs = sum(n * k for n, d, k in shapes)
        if self.opts is None:
            nb = int(load().gpa_gmm_batched_workspace_bytes(C.byref(arr), self.n_inst, self.chunk_points))
        else:
            nb = int(load().gpa_gmm_batched_workspace_bytes_opts(C.byref(arr), self.n_inst, C.byref(self.opts)))
        if nb == 0:
            raise GpaError(ERR_ARG, "gpa_gmm_batched_workspace_bytes")
        self.ws = workspace(nb, dev)

    def prepare(self, stream=None):
        if self.opts is None:
            rc = load().gmm_batched_prepare(C.byref(self.desc), self.n_inst, self.chunk_points, _ptr(self.ws),
                                            self.ws.numel(), _stream(stream))
        else:
            rc = load().gmm_batched_prepare_opts(C.byref(self.desc), self.n_inst, C.byref(self.opts),
                                                 _ptr(self.ws), self.ws.numel(), _stream(stream))
        _ok(rc, "gmm_batched_prepare")

    def run(self, ctas_per_sm=0, status=None, stream=None):
        if self.opts is None:
            rc = load().gmm_batched_vjp(C.byref(self.desc), self.n_inst, self.chunk_points, int(ctas_per_sm),
                                        _ptr(self.ws), self.ws.numel(), _ptr(status), _stream(stream))
        else:
            rc = load().gmm_batched_vjp_opts(C.byref(self.desc), self.n_inst, C.byref(self.opts), _ptr(self.ws),
                                             self.ws.numel(), _ptr(status), _stream(stream))
        _ok(rc, "gmm_batched_vjp")

    def zero_grads(self):
        self.flat.zero_()
        self.outs.zero_()

    def results(self):
        """[(objective, (d_alpha, d_mu, d_q, d_l))] per instance (device tensors)."""
        return [(out, tuple(g)) for _, g, out in self.tensors]


# ---------------------------------------------------------------------------
# Reprojection
# ---------------------------------------------------------------------------
def gpa_reproj_workspace_bytes(n_cams, n_pts, n_obs) -> int:
    return int(load().gpa_reproj_workspace_bytes(int(n_cams), int(n_pts), int(n_obs)))


def _reproj_params(cams, pts, obs):
    _check(cams, torch.float32, "cams")
    _check(pts, torch.float32, "pts")
    _check(obs, torch.int32, "obs")
    if cams.dim() != 2 or cams.shape[1] != 11:
        raise ValueError("cams must be [C, 11]")
    if pts.dim() != 2 or pts.shape[1] != 3:
        raise ValueError("pts must be [P, 3]")
    if obs.dim() != 2 or obs.shape[1] != 2:
        raise ValueError("obs must be [M, 2]")
    return cams.shape[0], pts.shape[0], obs.shape[0]


OBS_ORDERS = {"input": 0, "plan": 1}


def _obs_order(order):
    if order not in OBS_ORDERS:
        raise ValueError(f"obs_order must be 'input' or 'plan', got {order!r}")
    return OBS_ORDERS[order]


def reproj_residual(cams, pts, obs, tgt, res=None, plan=None, obs_order="input", ws=None, status=None,
                    stream=None):
    """res [M, 2] = projection - target; with a plan (gpa_obs_plan_build) the
    observations are visited in camera-sorted order (reproj_residual_sorted),
    and obs_order "plan" takes tgt and writes res in the plan's order."""
    order = _obs_order(obs_order)
    if order and plan is None:
        raise ValueError("obs_order 'plan' needs a plan")
    nc, npt, no = _reproj_params(cams, pts, obs)
    _check(tgt, torch.float32, "tgt", (no, 2))
    res = torch.empty(no, 2, dtype=torch.float32, device=cams.device) if res is None else res
    _check(res, torch.float32, "res", (no, 2))
    ws = workspace(gpa_reproj_workspace_bytes(nc, npt, no), cams.device) if ws is None else ws
    if plan is None:
        rc = load().reproj_residual(_ptr(cams), _ptr(pts), _ptr(obs), _ptr(tgt), nc, npt, no, _ptr(res), _ptr(ws),
                                    ws.numel(), _ptr(status), _stream(stream))
        _ok(rc, "reproj_residual")
    else:
        rc = load().reproj_residual_sorted(_ptr(cams), _ptr(pts), _ptr(obs), _ptr(tgt), nc, npt, no, _ptr(res),
                                           _ptr(plan), order, _ptr(ws), ws.numel(), _ptr(status), _stream(stream))
        _ok(rc, "reproj_residual_sorted")
    return res


def reproj_vjp(cams, pts, obs, w, d_cams=None, d_pts=None, strat="auto", plan=None, obs_order="input", ws=None,
               status=None, stream=None):
    """d_cams, d_pts += J^T w; obs_order "plan" (SORT) takes w in the plan's order."""
    order = _obs_order(obs_order)
    nc, npt, no = _reproj_params(cams, pts, obs)
    _check(w, torch.float32, "w", (no, 2))
    d_cams = torch.zeros(nc, 11, dtype=torch.float32, device=cams.device) if d_cams is None else d_cams
    d_pts = torch.zeros(npt, 3, dtype=torch.float32, device=cams.device) if d_pts is None else d_pts
    _check(d_cams, torch.float32, "d_cams", (nc, 11))
    _check(d_pts, torch.float32, "d_pts", (npt, 3))
    ws = workspace(gpa_reproj_workspace_bytes(nc, npt, no), cams.device) if ws is None else ws
    st = STRATEGIES[strat] if isinstance(strat, str) else int(strat)
    rc = load().reproj_vjp(_ptr(cams), _ptr(pts), _ptr(obs), _ptr(w), nc, npt, no, _ptr(d_cams), _ptr(d_pts), st,
                           _ptr(plan), order, _ptr(ws), ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "reproj_vjp")
    return d_cams, d_pts


def reproj_jvp(cams, pts, obs, v_cams, v_pts, jv=None, ws=None, status=None, stream=None):
    """J v per observation [M, 2] for tangents v_cams [C, 11], v_pts [P, 3]."""
    nc, npt, no = _reproj_params(cams, pts, obs)
    _check(v_cams, torch.float32, "v_cams", (nc, 11))
    _check(v_pts, torch.float32, "v_pts", (npt, 3))
    jv = torch.empty(no, 2, dtype=torch.float32, device=cams.device) if jv is None else jv
    _check(jv, torch.float32, "jv", (no, 2))
    ws = workspace(gpa_reproj_workspace_bytes(nc, npt, no), cams.device) if ws is None else ws
    rc = load().reproj_jvp(_ptr(cams), _ptr(pts), _ptr(obs), _ptr(v_cams), _ptr(v_pts), nc, npt, no, _ptr(jv),
                           _ptr(ws), ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "reproj_jvp")
    return jv


def reproj_normal_eqs(cams, pts, obs, tgt, U=None, V=None, W=None, g_cams=None, g_pts=None, res=None,
                      want_w=False, want_res=False, strat="auto", plan=None, w_order="input", ws=None, status=None,
                      stream=None):
    """Gauss-Newton blocks (U, V, W, g_cams, g_pts, res): U, V, g_cams, g_pts
    accumulate (+=, zeros if not given); W and res are written when given (or
    asked for with want_w / want_res), else None. W is [M][w_ld] with
    33 <= w_ld <= 64: J_c^T J_p in columns 0..32, zeros after (allocated with
    w_ld = 40, whole 32-byte sectors per row; take W[:, :33] for the blocks).
    w_order "input": row j is observation j; "plan" (with a plan): row i is
    the observation at position i of the plan's camera-sorted order."""
    if w_order not in ("input", "plan"):
        raise ValueError(f"w_order must be 'input' or 'plan', got {w_order!r}")
    nc, npt, no = _reproj_params(cams, pts, obs)
    _check(tgt, torch.float32, "tgt", (no, 2))
    dv = cams.device
    U = torch.zeros(nc, 66, device=dv) if U is None else _check(U, torch.float32, "U", (nc, 66))
    V = torch.zeros(npt, 6, device=dv) if V is None else _check(V, torch.float32, "V", (npt, 6))
    g_cams = torch.zeros(nc, 11, device=dv) if g_cams is None else _check(g_cams, torch.float32, "g_cams", (nc, 11))
    g_pts = torch.zeros(npt, 3, device=dv) if g_pts is None else _check(g_pts, torch.float32, "g_pts", (npt, 3))
    if W is None and want_w:
        W = torch.empty(no, 40, device=dv)
    w_ld = 0
    if W is not None:
        _check(W, torch.float32, "W")
        if W.dim() != 2 or W.shape[0] != no or not 33 <= W.shape[1] <= 64:
            raise ValueError(f"W must have shape ({no}, w_ld) with 33 <= w_ld <= 64, got {tuple(W.shape)}")
        w_ld = int(W.shape[1])
    if res is None and want_res:
        res = torch.empty(no, 2, device=dv)
    if res is not None:
        _check(res, torch.float32, "res", (no, 2))
    ws = workspace(int(load().gpa_reproj_gn_workspace_bytes(nc, npt, no)), dv) if ws is None else ws
    st = STRATEGIES[strat] if isinstance(strat, str) else int(strat)
    rc = load().reproj_normal_eqs(_ptr(cams), _ptr(pts), _ptr(obs), _ptr(tgt), nc, npt, no, _ptr(U), _ptr(V),
                                  _ptr(W), w_ld, 1 if w_order == "plan" else 0, _ptr(g_cams), _ptr(g_pts),
                                  _ptr(res), st, _ptr(plan), _ptr(ws),
                                  ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "reproj_normal_eqs")
    return U, V, W, g_cams, g_pts, res


def gpa_check_bounded_wait(limit_ns, status, gave_up, stream=None):
    """Launch the device-wait check: 64 threads wait on an mbarrier nobody
    arrives at and give up after limit_ns (status |= GPA_ERR_TIMEOUT, gave_up
    += 1 per thread). status and gave_up: zeroed int32 device tensors."""
    _check(status, torch.int32, "status", (1,))
    _check(gave_up, torch.int32, "gave_up", (1,))
    rc = load().gpa_check_bounded_wait(int(limit_ns), _ptr(status), _ptr(gave_up), _stream(stream))
    _ok(rc, "gpa_check_bounded_wait")


def reproj_vjp_noalloc(cams, pts, obs, w, d_cams=None, d_pts=None, strat="auto", plan=None, status=None,
                       stream=None):
    """reproj_vjp without a workspace: the camera scratch is the library's own
    fixed device array (at most GPA_NOALLOC_MAX_CAMS = 16384 cameras)."""
    nc, npt, no = _reproj_params(cams, pts, obs)
    _check(w, torch.float32, "w", (no, 2))
    d_cams = torch.zeros(nc, 11, dtype=torch.float32, device=cams.device) if d_cams is None else d_cams
    d_pts = torch.zeros(npt, 3, dtype=torch.float32, device=cams.device) if d_pts is None else d_pts
    _check(d_cams, torch.float32, "d_cams", (nc, 11))
    _check(d_pts, torch.float32, "d_pts", (npt, 3))
    st = STRATEGIES[strat] if isinstance(strat, str) else int(strat)
    rc = load().reproj_vjp_noalloc(_ptr(cams), _ptr(pts), _ptr(obs), _ptr(w), nc, npt, no, _ptr(d_cams), _ptr(d_pts),
                                   st, _ptr(plan), _ptr(status), _stream(stream))
    _ok(rc, "reproj_vjp_noalloc")
    return d_cams, d_pts


def reproj_residual_vjp(cams, pts, obs, tgt, wscale=1.0, res=None, d_cams=None, d_pts=None, strat="auto",
                        plan=None, obs_order="input", ws=None, status=None, stream=None):
    """res and d_cams, d_pts += J^T (wscale res) in one pass; obs_order "plan"
    (SORT) takes tgt and writes res in the plan's order."""
    order = _obs_order(obs_order)
    nc, npt, no = _reproj_params(cams, pts, obs)
    _check(tgt, torch.float32, "tgt", (no, 2))
    res = torch.empty(no, 2, dtype=torch.float32, device=cams.device) if res is None else res
    d_cams = torch.zeros(nc, 11, dtype=torch.float32, device=cams.device) if d_cams is None else d_cams
    d_pts = torch.zeros(npt, 3, dtype=torch.float32, device=cams.device) if d_pts is None else d_pts
    ws = workspace(gpa_reproj_workspace_bytes(nc, npt, no), cams.device) if ws is None else ws
    st = STRATEGIES[strat] if isinstance(strat, str) else int(strat)
    rc = load().reproj_residual_vjp(_ptr(cams), _ptr(pts), _ptr(obs), _ptr(tgt), nc, npt, no, float(wscale),
                                    _ptr(res), _ptr(d_cams), _ptr(d_pts), st, _ptr(plan), order, _ptr(ws),
                                    ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "reproj_residual_vjp")
    return res, d_cams, d_pts


# ---------------------------------------------------------------------------
# Plans and the generic scatter
# ---------------------------------------------------------------------------
def gpa_plan_bytes(n, n_keys) -> int:
    return int(load().gpa_plan_bytes(int(n), int(n_keys)))


def gpa_plan_workspace_bytes(n, n_keys) -> int:
    return int(load().gpa_plan_workspace_bytes(int(n), int(n_keys)))


def gpa_obs_plan_build(obs, n_cams, n_pts, plan=None, ws=None, status=None, stream=None):
    _check(obs, torch.int32, "obs")
    no = obs.shape[0]
    plan = workspace(gpa_plan_bytes(no, n_cams), obs.device) if plan is None else plan
    ws = workspace(gpa_plan_workspace_bytes(no, n_cams), obs.device) if ws is None else ws
    rc = load().gpa_obs_plan_build(_ptr(obs), no, int(n_cams), int(n_pts), _ptr(plan), plan.numel(), _ptr(ws),
                                   ws.numel(), _ptr(status), _stream(stream))
    _ok(rc, "gpa_obs_plan_build")
    return plan


def gpa_index_plan_build(idx, n_keys, plan=None, ws=None, status=None, stream=None):
    _check(idx, torch.int32, "idx")
    m = idx.shape[0]
    plan = workspace(gpa_plan_bytes(m, n_keys), idx.device) if plan is None else plan
    ws = workspace(gpa_plan_workspace_bytes(m, n_keys), idx.device) if ws is None else ws
    rc = load().gpa_index_plan_build(_ptr(idx), m, int(n_keys), _ptr(plan), plan.numel(), _ptr(ws), ws.numel(),
                                     _ptr(status), _stream(stream))
    _ok(rc, "gpa_index_plan_build")
    return plan


def plan_arrays(plan, n, n_keys):
    """Views (header, perm, key_sorted, aux_sorted, seg_off) into a plan buffer."""
    def a256(v):
        return (v + 255) & ~255
    off = 256
    hdr = plan[:32].view(torch.int64)
    arrs = []
    for _ in range(3):
        arrs.append(plan[off:off + 4 * n].view(torch.int32))
        off += a256(4 * n)
    seg = plan[off:off + 4 * (n_keys + 1)].view(torch.int32)
    return hdr, arrs[0], arrs[1], arrs[2], seg


def accum_scatter_add(idx, vals, acc, strat="auto", plan=None, status=None, stream=None):
    _check(idx, torch.int32, "idx")
    m = idx.shape[0]
    if vals.dtype not in (torch.float32, torch.int32) or acc.dtype != vals.dtype:
        raise TypeError("vals and acc must both be float32 or both int32")
    _check(vals, vals.dtype, "vals")
    _check(acc, acc.dtype, "acc")
    w = 1 if vals.dim() == 1 else vals.shape[1]
    if vals.shape[0] != m:
        raise ValueError("vals must have one row per index")
    nb = acc.shape[0]
    st = STRATEGIES[strat] if isinstance(strat, str) else int(strat)
    dtype = 0 if vals.dtype == torch.float32 else 1
    rc = load().accum_scatter_add(_ptr(idx), _ptr(vals), m, w, dtype, _ptr(acc), nb, st, _ptr(plan), _ptr(status),
                                  _stream(stream))
    _ok(rc, "accum_scatter_add")
    return acc
