"""Python face of the C ABI: argument marshalling only.

Tensors are passed to the library as raw pointers; every computation runs in
the CUDA library.  Device tensors (torch, on the handle's device) are used in
place; numpy arrays are passed as host pointers and the library stages them.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

try:  # torch is plumbing only: device memory and streams
    import torch
except Exception:  # pragma: no cover
    torch = None


def _ptr(a):
    if a is None:
        return None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _dtype_of(prec: str):
    return "float64" if prec == "fp64" else "float32"


def _check_dtype(a, prec, name):
    want = _dtype_of(prec)
    got = str(a.dtype).replace("torch.", "")
    if got != want:
        raise TypeError(f"{name} must be {want} for precision {prec} (got {got})")


def param_permutation(widths) -> np.ndarray:
    lib = _lib.load()
    w = (ctypes.c_int * len(widths))(*widths)
    P = sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1))
    out = np.empty(P, dtype=np.int64)
    _lib.check(lib.hess_param_permutation(len(widths), w,
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


class HessMLP:
    """Handle on a network and a parameter point (hess_mlp_create)."""

    def __init__(self, widths, acts, omega, stream=None):
        self._lib = _lib.load()
        self.widths = [int(t) for t in widths]
        self.acts = list(acts)
        w = (ctypes.c_int * len(self.widths))(*self.widths)
        a = (ctypes.c_int * max(1, len(self.acts)))(*[_lib.ACT[x] for x in self.acts] or [0])
        desc = _lib.HessDesc(len(self.widths), w, a)
        self._keep = (w, a)
        if isinstance(omega, np.ndarray):
            omega = np.ascontiguousarray(omega, dtype=np.float64)
        h = ctypes.c_void_p()
        _lib.check(self._lib.hess_mlp_create(ctypes.byref(desc), _ptr(omega),
                                             ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        self.P = int(self._lib.hess_mlp_num_params(self.h))

    def close(self):
        if getattr(self, "h", None):
            self._lib.hess_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, omega):
        if isinstance(omega, np.ndarray):
            omega = np.ascontiguousarray(omega, dtype=np.float64)
        _lib.check(self._lib.hess_mlp_set_params(self.h, _ptr(omega)))

    def set_stream(self, stream):
        _lib.check(self._lib.hess_mlp_set_stream(self.h, ctypes.c_void_p(stream or 0)))

    def set_operand_limit(self, nbytes: int):
        _lib.check(self._lib.hess_mlp_set_operand_limit(self.h, int(nbytes)))

    def set_eig_blocks(self, blocks: int):
        _lib.check(self._lib.hess_mlp_set_eig_blocks(self.h, int(blocks)))

    def timing(self, enable: bool):
        _lib.check(self._lib.hess_timing_enable(self.h, 1 if enable else 0))

    def read_timing(self, kernel_class: str) -> dict:
        st = _lib.KernelStats()
        _lib.check(self._lib.hess_timing_read(self.h, _lib.KERNEL_CLASS[kernel_class],
                                              ctypes.byref(st)))
        return {"launches": st.launches, "ms": st.ms, "flops": st.flops, "bytes": st.bytes, "sm_ms": st.sm_ms}

    # ------------------------------------------------------------ calls
    def _io(self, X, Y, prec):
        _check_dtype(X, prec, "X")
        _check_dtype(Y, prec, "Y")
        return int(X.shape[0])

    def per_example_grads(self, X, Y, prec="fp64", out=None):
        N = self._io(X, Y, prec)
        out = self._alloc_like(X, (N, self.P), prec) if out is None else out
        _lib.check(self._lib.per_example_grads(self.h, _ptr(X), _ptr(Y), N,
                                               _lib.PRECISION[prec], _ptr(out)))
        return out

    def opg(self, X, Y, prec="fp64", out=None):
        N = self._io(X, Y, prec)
        out = self._alloc_like(X, (self.P, self.P), prec) if out is None else out
        _lib.check(self._lib.opg(self.h, _ptr(X), _ptr(Y), N, _lib.PRECISION[prec], _ptr(out)))
        return out

    def exact_hessian(self, X, Y, prec="fp64", out=None):
        N = self._io(X, Y, prec)
        out = self._alloc_like(X, (self.P, self.P), prec) if out is None else out
        _lib.check(self._lib.exact_hessian(self.h, _ptr(X), _ptr(Y), N, _lib.PRECISION[prec],
                                           _ptr(out)))
        return out

    def opg_topk_eig(self, X, Y, k, prec="fp64", evals=None, evecs=None, allow_deficient=False):
        """Returns (evals (k,), evecs (k, P) whose row c is q_c, status)."""
        N = self._io(X, Y, prec)
        if evals is None:
            evals = self._alloc_like(X, (k,), "fp64")
        if evecs is None:
            evecs = self._alloc_like(X, (k, self.P), "fp64")
        allow = (_lib.HESS_ERR_RANK_DEFICIENT,) if allow_deficient else ()
        st = _lib.check(self._lib.opg_topk_eig(self.h, _ptr(X), _ptr(Y), N, int(k),
                                               _lib.PRECISION[prec], _ptr(evals), _ptr(evecs)),
                        allow)
        return evals, evecs, st

    def hvp(self, X, Y, V, prec="fp64", out=None):
        """H v for the rows v of V (b x P, or one P-vector); returns the
        products in the same shape (hessian_vector_products)."""
        N = self._io(X, Y, prec)
        _check_dtype(V, prec, "V")
        b = 1 if len(V.shape) == 1 else int(V.shape[0])
        if int(V.shape[-1]) != self.P:
            raise ValueError(f"directions must have P = {self.P} entries")
        out = self._alloc_like(X, tuple(V.shape), prec) if out is None else out
        _lib.check(self._lib.hessian_vector_products(self.h, _ptr(X), _ptr(Y), N,
                                                     _lib.PRECISION[prec], _ptr(V), b, _ptr(out)))
        return out

    def hessian_topk_eig(self, X, Y, k, prec="fp64", evals=None, evecs=None):
        """Top-k eigenpairs of the exact Hessian by Lanczos on H v products.
        Returns (evals (k,), evecs (k, P) whose row c is q_c, Krylov steps)."""
        N = self._io(X, Y, prec)
        if evals is None:
            evals = self._alloc_like(X, (k,), "fp64")
        if evecs is None:
            evecs = self._alloc_like(X, (k, self.P), "fp64")
        steps = ctypes.c_int(0)
        _lib.check(self._lib.hessian_topk_eig(self.h, _ptr(X), _ptr(Y), N, int(k),
                                              _lib.PRECISION[prec], _ptr(evals), _ptr(evecs),
                                              ctypes.byref(steps)))
        return evals, evecs, steps.value

    def opg_topk_eig_streaming(self, X, Y, k, prec="fp64", chunk=8192, evals=None, evecs=None,
                               allow_deficient=False):
        """Top-k OPG eigenpairs from chunks of examples (P x P FP64 sum, no
        Gram matrix).  Returns (evals (k,), evecs (k, P), status)."""
        N = self._io(X, Y, prec)
        if evals is None:
            evals = self._alloc_like(X, (k,), "fp64")
        if evecs is None:
            evecs = self._alloc_like(X, (k, self.P), "fp64")
        allow = (_lib.HESS_ERR_RANK_DEFICIENT,) if allow_deficient else ()
        st = _lib.check(self._lib.opg_topk_eig_streaming(self.h, _ptr(X), _ptr(Y), N, int(k),
                                                         _lib.PRECISION[prec], int(chunk), _ptr(evals),
                                                         _ptr(evecs)), allow)
        return evals, evecs, st

    def hessian_minibatches(self, X, Y, bs, prec="fp64", out=None):
        """Mini-batch Hessians of consecutive batches of bs examples (bs = 1:
        per-example Hessians); returns an array (ceil(N / bs), P, P)."""
        N = self._io(X, Y, prec)
        nb = -(-N // max(int(bs), 1))
        out = self._alloc_like(X, (nb, self.P, self.P), prec) if out is None else out
        _lib.check(self._lib.hessian_minibatches(self.h, _ptr(X), _ptr(Y), N, int(bs),
                                                 _lib.PRECISION[prec], _ptr(out)))
        return out

    def approx_form(self, evals, evecs, full=False, lam_tilde=float("nan"), prec="fp64", out=None):
        """The low-rank (Sec. 4.1) or full-rank (Sec. 4.2) approximation from K
        eigenpairs (evecs: K x P, row c = q_c), formed as a P x P matrix."""
        K = int(evals.shape[0])
        if tuple(evecs.shape) != (K, self.P):
            raise ValueError(f"evecs must be {K} x {self.P}")
        out = self._alloc_like(evecs, (self.P, self.P), prec) if out is None else out
        _lib.check(self._lib.hess_approx_form(self.h, K, _ptr(evals), _ptr(evecs), 1 if full else 0,
                                              float(lam_tilde), _lib.PRECISION[prec], _ptr(out)))
        return out

    def approx_apply(self, evals, evecs, X, full=False, lam_tilde=float("nan"), products=True):
        """For each row x of X (b x P, float64): (H~ x rows or None, x^T H~ x)
        without forming H~ (Sec. 5.5, 5.6)."""
        K = int(evals.shape[0])
        b = 1 if len(X.shape) == 1 else int(X.shape[0])
        _check_dtype(X, "fp64", "X")
        HX = self._alloc_like(X, tuple(X.shape), "fp64") if products else None
        quad = self._alloc_like(X, (b,), "fp64")
        _lib.check(self._lib.hess_approx_apply(self.h, K, _ptr(evals), _ptr(evecs), 1 if full else 0,
                                               float(lam_tilde), _ptr(X), b, _ptr(HX), _ptr(quad)))
        return HX, quad

    def curvature(self, X, Y, prec="bf16x3", opg=None, hessian=None, k=0, evals=None, evecs=None,
                  allow_deficient=False):
        """OPG, exact Hessian and top-k eigenpairs in one call (hess_curvature);
        the given output buffers are filled.  Returns the status."""
        N = self._io(X, Y, prec)
        allow = (_lib.HESS_ERR_RANK_DEFICIENT,) if allow_deficient else ()
        return _lib.check(self._lib.hess_curvature(self.h, _ptr(X), _ptr(Y), N, _lib.PRECISION[prec],
                                                   _ptr(opg), _ptr(hessian), int(k), _ptr(evals),
                                                   _ptr(evecs)), allow)

    @staticmethod
    def _alloc_like(X, shape, prec):
        dt = _dtype_of(prec)
        if torch is not None and isinstance(X, torch.Tensor):
            return torch.empty(shape, dtype=getattr(torch, dt), device=X.device)
        return np.empty(shape, dtype=dt)


def autotune(enable: bool = True):
    """Turn tile-width autotuning of the tensor-core contractions on or off."""
    _lib.check(_lib.load().hess_autotune(1 if enable else 0))


def autotune_entries() -> int:
    return int(_lib.load().hess_autotune_entries())


def autotune_save(path: str):
    _lib.check(_lib.load().hess_autotune_save(str(path).encode()))


def autotune_load(path: str):
    _lib.check(_lib.load().hess_autotune_load(str(path).encode()))


class HessBatch:
    """Batched OPG / exact Hessian of many networks (hess_batch_*): marshalling only."""

    def __init__(self, workspace_bytes=16 << 30, stream=None):
        self._lib = _lib.load()
        b = ctypes.c_void_p()
        _lib.check(self._lib.hess_batch_create(int(workspace_bytes), ctypes.c_void_p(stream or 0),
                                               ctypes.byref(b)))
        self.b = b

    def run(self, items, prec="bf16x3"):
        """items: sequence of (HessMLP, X, Y, opg_out or None, hessian_out or None) with
        device float32 tensors.  Returns the wave statistics as a dict."""
        arr = (_lib.BatchItem * max(1, len(items)))()
        for i, (net, X, Y, o, hs) in enumerate(items):
            arr[i] = _lib.BatchItem(net.h, _ptr(X), _ptr(Y), int(X.shape[0]), _ptr(o), _ptr(hs))
        info = _lib.BatchInfo()
        _lib.check(self._lib.hess_batch_run(self.b, arr, len(items), _lib.PRECISION[prec],
                                            ctypes.byref(info)))
        return {"waves": info.waves, "items_chunked": info.items_chunked, "tiles": info.tiles,
                "flops": info.flops, "launch_ms": info.launch_ms,
                "graph_replayed": bool(info.graph_replayed)}

    def set_graphs(self, enable: bool):
        """Capture repeated runs of the same item list in a CUDA graph."""
        _lib.check(self._lib.hess_batch_set_graphs(self.b, 1 if enable else 0))

    def close(self):
        if getattr(self, "b", None):
            self._lib.hess_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HessServer:
    """Continuous-batching request server (hess_server_*): marshalling only."""

    def __init__(self, slots=4, budget_bytes=100 << 30):
        self._lib = _lib.load()
        s = ctypes.c_void_p()
        _lib.check(self._lib.hess_server_create(int(slots), int(budget_bytes), ctypes.byref(s)))
        self.s = s
        self._keep = {}

    def add_network(self, widths, acts, omega):
        w = (ctypes.c_int * len(widths))(*[int(t) for t in widths])
        a = (ctypes.c_int * max(1, len(acts)))(*([_lib.ACT[x] for x in acts] or [0]))
        desc = _lib.HessDesc(len(widths), w, a)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        nid = ctypes.c_int()
        _lib.check(self._lib.hess_server_add_network(self.s, ctypes.byref(desc), _ptr(omega),
                                                     ctypes.byref(nid)))
        return nid.value

    def submit(self, kind, net, X, Y, prec, out, k=0, evals=None):
        """Queue a request; X, Y, out (and evals) must stay alive until wait()."""
        r = _lib.HessRequest(_lib.REQUEST_KIND[kind], int(net), _ptr(X), _ptr(Y), int(X.shape[0]),
                             _lib.PRECISION[prec], int(k), _ptr(out),
                             ctypes.cast(_ptr(evals), ctypes.POINTER(ctypes.c_double))
                             if evals is not None else None)
        t = ctypes.c_int64()
        _lib.check(self._lib.hess_server_submit(self.s, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (X, Y, out, evals)
        return t.value

    def wait(self, ticket, timeout=-1.0):
        """Returns the request's status (raises on a wait timeout)."""
        res = ctypes.c_int()
        _lib.check(self._lib.hess_server_wait(self.s, int(ticket), float(timeout), ctypes.byref(res)))
        self._keep.pop(ticket, None)
        return res.value

    def wait_timed(self, ticket, timeout=-1.0):
        """Returns (status, gpu_start_ms, gpu_end_ms): the request's device
        interval in ms since the server was created."""
        res = ctypes.c_int()
        a, b = ctypes.c_double(), ctypes.c_double()
        _lib.check(self._lib.hess_server_wait_timed(self.s, int(ticket), float(timeout), ctypes.byref(res),
                                                    ctypes.byref(a), ctypes.byref(b)))
        self._keep.pop(ticket, None)
        return res.value, a.value, b.value

    def close(self):
        if getattr(self, "s", None):
            self._lib.hess_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
