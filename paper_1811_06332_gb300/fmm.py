"""ctypes binding of libfmm_gb300.so (C-ABI declared in include/fmm_gb300.h).

Argument marshalling only: every function forwards device pointers (taken
from torch tensors) and sizes to the entry point of the same name; all the
arithmetic runs in the library's CUDA kernels.  Loading fails loudly when the
library has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmm_gb300.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_STATE, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
BASIS_SYM, BASIS_TRACELESS, BASIS_TG = 0, 1, 2
FP64, FP32, GEMM_TF32X3, GEMM_BF16X3 = 0, 1, 2, 3

EXPORTS = [
    "fmm_ncoef", "fmm_create", "fmm_destroy", "fmm_last_error", "fmm_build_tree", "fmm_p2m", "fmm_m2m",
    "fmm_m2l", "fmm_m2l_levels", "fmm_tc_layout", "fmm_tc_gen_layout", "fmm_l2l", "fmm_l2p", "fmm_p2p", "fmm_evaluate",
    "fmm_evaluate_host", "fmm_evaluate_dipoles", "fmm_op_dtensor",
    "fmm_op_p2m", "fmm_op_m2m", "fmm_op_m2m_fused", "fmm_m2m_fused_terms", "fmm_op_m2l", "fmm_op_l2l", "fmm_op_l2p", "fmm_direct",
    "fmm_kernel_launches", "fmm_evaluate_noalloc", "fmm_sync_status", "fmm_selftest_wait", "fmm_l2p_p2p", "fmm_plan_stats", "fmm_plan_pairs", "fmm_pair_data",
    "fmm_mlp_grad", "fmm_mlp_train", "fmm_mlp_predict", "fmm_set_mlp", "fmm_set_pair_orders",
    "fmm_plan_pair_orders", "fmm_set_tc_shape", "fmm_plan_tuning", "fmm_tune_cache_get", "fmm_tune_cache_put",
]

MLP_NF, MLP_NOUT, MLP_NBLOB = 12, 9, 9769


class FMMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fmm status %d: %s" % (code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("basis", ctypes.c_int), ("prec", ctypes.c_int),
                ("adaptive", ctypes.c_int), ("depth", ctypes.c_int), ("max_leaf", ctypes.c_int),
                ("theta", ctypes.c_double), ("learned_p", ctypes.c_int),
                ("target_rel_err", ctypes.c_double), ("use_graph", ctypes.c_int), ("autotune", ctypes.c_int),
                ("ap", ctypes.c_int),
                ("binary_tree", ctypes.c_int)]


_lib = None
_vp, _i64, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfmm_gb300.so is not built (run __graft_entry__.build()); "
                               "the CUDA library is required, there is no CPU path")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "fmm_ncoef": ([_int, _int], _int),
            "fmm_create": ([ctypes.POINTER(Config), ctypes.POINTER(_vp)], _int),
            "fmm_destroy": ([_vp], None),
            "fmm_last_error": ([_vp], ctypes.c_char_p),
            "fmm_build_tree": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp], _int),
            "fmm_p2m": ([_vp, _vp], _int), "fmm_m2m": ([_vp, _vp], _int),
            "fmm_m2l": ([_vp, _vp], _int), "fmm_m2l_levels": ([_vp, _int, _int, _vp], _int),
            "fmm_tc_layout": ([_int, _int, _vp, _int], _int),
            "fmm_tc_gen_layout": ([_int, _int, _int, _vp, _int, _vp, _int], _int),
            "fmm_l2l": ([_vp, _vp], _int),
            "fmm_l2p": ([_vp, _vp, _vp, _vp, _vp, _vp], _int),
            "fmm_p2p": ([_vp, _vp, _vp, _vp, _vp, _vp], _int),
            "fmm_l2p_p2p": ([_vp, _vp, _vp, _vp, _vp, _vp], _int),
            "fmm_evaluate": ([_vp, _i64] + [_vp] * 9, _int),
            "fmm_evaluate_host": ([_vp, _i64] + [_vp] * 9, _int),
            "fmm_evaluate_dipoles": ([_vp, _i64] + [_vp] * 12, _int),
            "fmm_op_dtensor": ([_int, _int, _int, _i64, _vp, _vp, _vp], _int),
            "fmm_op_p2m": ([_int, _int, _i64] + [_vp] * 8, _int),
            "fmm_op_m2m": ([_int, _int, _int, _i64, _vp, _vp, _vp, _vp], _int),
            "fmm_op_m2m_fused": ([_int, _i64, _vp, _vp, _vp, _vp], _int),
            "fmm_m2m_fused_terms": ([_int], _int),
            "fmm_op_m2l": ([_int, _int, _int, _i64, _vp, _vp, _vp, _int, _vp], _int),
            "fmm_op_l2l": ([_int, _int, _int, _i64, _vp, _vp, _vp, _vp], _int),
            "fmm_op_l2p": ([_int, _int, _int, _i64, _vp, _vp, _vp, _vp], _int),
            "fmm_sync_status": ([_vp, _vp], _int),
            "fmm_selftest_wait": ([ctypes.c_int64, _int, _vp], _int),
            "fmm_direct": ([_i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp], _int),
            "fmm_kernel_launches": ([], _i64),
            "fmm_evaluate_noalloc": ([_int, _int, _int, _i64] + [_vp] * 9, _int),
            "fmm_plan_stats": ([_vp, _vp, _int], _int),
            "fmm_plan_pairs": ([_vp, _vp, _vp, _i64, _vp], _int),
            "fmm_pair_data": ([_vp, _vp, _vp, _vp], _int),
            "fmm_mlp_grad": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp], _int),
            "fmm_mlp_train": ([_vp, _i64, _vp, _vp, _vp, _int, _int, ctypes.c_float, _int, _vp, _vp], _int),
            "fmm_mlp_predict": ([_vp, _i64, _vp, _vp, _vp], _int),
            "fmm_set_mlp": ([_vp, _vp, _i64], _int),
            "fmm_set_pair_orders": ([_vp, _vp, _i64], _int),
            "fmm_plan_pair_orders": ([_vp, _vp, _i64, _vp], _int),
            "fmm_set_tc_shape": ([_vp, _int, _int], _int),
            "fmm_plan_tuning": ([_vp, _vp, _int], _int),
            "fmm_tune_cache_get": ([ctypes.c_char_p, ctypes.c_char_p, _vp], _int),
            "fmm_tune_cache_put": ([ctypes.c_char_p, ctypes.c_char_p, _vp, ctypes.c_double], _int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if t.is_cuda and not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _check(rc, plan=None):
    if rc != OK:
        msg = lib().fmm_last_error(plan)
        raise FMMError(rc, msg.decode() if msg else "")
    return rc


def ncoef(p: int, basis: int) -> int:
    n = lib().fmm_ncoef(p, basis)
    if n < 0:
        raise FMMError(n, "bad p/basis")
    return n


def kernel_launches() -> int:
    return lib().fmm_kernel_launches()


# ---------------------------------------------------------------------------
# operator-level calls (device tensors, physical units)
# ---------------------------------------------------------------------------
def fmm_op_dtensor(p, prec, r, D, basis=BASIS_SYM, stream=None):
    _check(lib().fmm_op_dtensor(p, basis, prec, r.shape[1], _ptr(r), _ptr(D), _stream(stream)))


def fmm_op_p2m(p, basis, start, x, y, z, q, centre, M, stream=None):
    _check(lib().fmm_op_p2m(p, basis, len(start) - 1, _ptr(start), _ptr(x), _ptr(y), _ptr(z), _ptr(q),
                            _ptr(centre), _ptr(M), _stream(stream)))


def _prec_of(t):
    return FP32 if t.dtype == torch.float32 else FP64


def fmm_op_m2m(p, basis, Mc, delta, Mp, stream=None):
    """FP64 or FP32 by the dtype of Mc (Mp must match)."""
    _check(lib().fmm_op_m2m(p, basis, _prec_of(Mc), Mc.shape[1], _ptr(Mc), _ptr(delta), _ptr(Mp),
                            _stream(stream)))


def fmm_op_m2m_fused(p, Mc, delta, Mp, stream=None):
    """Fused traceless M2M (Eq. Detracer2), FP64, traceless storage."""
    _check(lib().fmm_op_m2m_fused(p, Mc.shape[1], _ptr(Mc), _ptr(delta), _ptr(Mp), _stream(stream)))


def fmm_op_m2l(p, basis, prec, M, r, L, accumulate=False, stream=None):
    _check(lib().fmm_op_m2l(p, basis, prec, M.shape[1], _ptr(M), _ptr(r), _ptr(L), int(accumulate),
                            _stream(stream)))


def fmm_op_l2l(p, basis, Lp, delta, Lc, stream=None):
    """FP64 or FP32 by the dtype of Lp (Lc must match)."""
    _check(lib().fmm_op_l2l(p, basis, _prec_of(Lp), Lp.shape[1], _ptr(Lp), _ptr(delta), _ptr(Lc),
                            _stream(stream)))


def fmm_op_l2p(p, basis, L, rb, out, stream=None):
    """FP64 or FP32 by the dtype of L (out must match)."""
    _check(lib().fmm_op_l2p(p, basis, _prec_of(L), L.shape[1], _ptr(L), _ptr(rb), _ptr(out), _stream(stream)))


def _host_f32(blob):
    import numpy as np
    b = np.ascontiguousarray(blob, dtype=np.float32)
    if b.shape != (MLP_NBLOB,):
        raise ValueError("blob must hold %d floats" % MLP_NBLOB)
    return b


def fmm_mlp_grad(blob, feat, labels, stream=None):
    """Loss and gradient (numpy, FP32) of the order model over the samples
    (device float32 feat [n, 12], labels [n, 9])."""
    import numpy as np
    b = _host_f32(blob)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(MLP_NBLOB - 2 * MLP_NF - 8, dtype=np.float32)
    _check(lib().fmm_mlp_grad(b.ctypes.data, feat.shape[0], _ptr(feat), _ptr(labels), loss.ctypes.data,
                              grad.ctypes.data, _stream(stream)))
    return float(loss[0]), grad


def fmm_mlp_train(blob, feat, labels, order, epochs, batch, lr, fit_moments=True, stream=None):
    """Trains in place on a copy of blob; returns (trained blob, per-epoch loss)."""
    import numpy as np
    b = _host_f32(blob).copy()
    losses = np.zeros(max(epochs, 1), dtype=np.float32)
    _check(lib().fmm_mlp_train(b.ctypes.data, feat.shape[0], _ptr(feat), _ptr(labels), _ptr(order), epochs, batch,
                               float(lr), int(fit_moments), losses.ctypes.data, _stream(stream)))
    return b, losses[:epochs]


def fmm_mlp_predict(blob, feat, pred, stream=None):
    b = _host_f32(blob)
    _check(lib().fmm_mlp_predict(b.ctypes.data, feat.shape[0], _ptr(feat), _ptr(pred), _stream(stream)))


def fmm_selftest_wait(spin, arrive, stream=None):
    """Bounded-wait self-test (fmm_selftest_wait): FMM_OK when the barrier is
    arrived on; raises FMMError (FMM_ERR_TIMEOUT) when the wait gives up."""
    _check(lib().fmm_selftest_wait(int(spin), int(arrive), _stream(stream)))


def fmm_direct(x, y, z, q, pot, ax, ay, az, targets=None, stream=None):
    nt = len(targets) if targets is not None else len(x)
    _check(lib().fmm_direct(len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(q), nt, _ptr(targets), _ptr(pot),
                            _ptr(ax), _ptr(ay), _ptr(az), _stream(stream)))


# ---------------------------------------------------------------------------
# plan
# ---------------------------------------------------------------------------
class Plan:
    """Owns an fmm_plan (uniform octree FMM of App. C)."""

    def __init__(self, p, basis=BASIS_SYM, prec=FP64, depth=3, use_graph=False, adaptive=False,
                 max_leaf=64, theta=0.5, learned_p=False, target_rel_err=1e-4, autotune=False, ap=False,
                 binary_tree=False):
        cfg = Config(p=p, basis=basis, prec=prec, adaptive=int(adaptive), depth=depth, max_leaf=max_leaf,
                     theta=theta, learned_p=int(learned_p), target_rel_err=target_rel_err,
                     use_graph=int(use_graph), autotune=int(autotune), ap=int(ap),
                     binary_tree=int(binary_tree))
        h = _vp()
        _check(lib().fmm_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.cfg = cfg

    def close(self):
        if self.h:
            lib().fmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        return _check(rc, self.h)

    def fmm_build_tree(self, x, y, z, q, stream=None):
        self._c(lib().fmm_build_tree(self.h, len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(q), _stream(stream)))

    def fmm_p2m(self, stream=None):
        self._c(lib().fmm_p2m(self.h, _stream(stream)))

    def fmm_m2m(self, stream=None):
        self._c(lib().fmm_m2m(self.h, _stream(stream)))

    def fmm_m2l(self, stream=None):
        self._c(lib().fmm_m2l(self.h, _stream(stream)))

    def fmm_m2l_levels(self, lmin, lmax, stream=None):
        self._c(lib().fmm_m2l_levels(self.h, int(lmin), int(lmax), _stream(stream)))

    def fmm_l2l(self, stream=None):
        self._c(lib().fmm_l2l(self.h, _stream(stream)))

    def fmm_l2p(self, pot, ax, ay, az, stream=None):
        self._c(lib().fmm_l2p(self.h, _ptr(pot), _ptr(ax), _ptr(ay), _ptr(az), _stream(stream)))

    def fmm_p2p(self, pot, ax, ay, az, stream=None):
        self._c(lib().fmm_p2p(self.h, _ptr(pot), _ptr(ax), _ptr(ay), _ptr(az), _stream(stream)))

    def fmm_l2p_p2p(self, pot, ax, ay, az, stream=None):
        self._c(lib().fmm_l2p_p2p(self.h, _ptr(pot), _ptr(ax), _ptr(ay), _ptr(az), _stream(stream)))

    def fmm_evaluate(self, x, y, z, q, pot, ax, ay, az, stream=None):
        self._c(lib().fmm_evaluate(self.h, len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(q), _ptr(pot), _ptr(ax),
                                   _ptr(ay), _ptr(az), _stream(stream)))

    def fmm_evaluate_dipoles(self, x, y, z, q, px, py, pz, pot, ax, ay, az, stream=None):
        self._c(lib().fmm_evaluate_dipoles(self.h, len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(q), _ptr(px), _ptr(py),
                                           _ptr(pz), _ptr(pot), _ptr(ax), _ptr(ay), _ptr(az), _stream(stream)))

    def fmm_evaluate_host(self, x, y, z, q, pot, ax, ay, az, stream=None):
        """Host (CPU) tensors or numpy arrays of float64; synchronous."""
        import numpy as np

        def hp(a):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
                return a.ctypes.data
            assert not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
            return a.data_ptr()
        self._c(lib().fmm_evaluate_host(self.h, len(x), hp(x), hp(y), hp(z), hp(q), hp(pot), hp(ax), hp(ay),
                                        hp(az), _stream(stream)))

    def sync_status(self, stream=None):
        """Waits for the stream; raises FMMError (FMM_ERR_TIMEOUT) if a bounded
        device wait of the plan's tensor-core kernels gave up since the last check."""
        self._c(lib().fmm_sync_status(self.h, _stream(stream)))

    def set_tc_shape(self, kernel, cw):
        self._c(lib().fmm_set_tc_shape(self.h, int(kernel), int(cw)))

    def tuning(self):
        """Tensor-core kernel shape in use and the autotuner's candidates."""
        import numpy as np
        v = np.zeros(5 + 4 * 8, dtype=np.int32)
        n = lib().fmm_plan_tuning(self.h, v.ctypes.data, len(v))
        if n < 0:
            _check(n)
        cand = [dict(zip(("kernel", "cw", "niss", "us"), v[5 + 4 * c:9 + 4 * c].tolist())) for c in range(v[4])]
        return {"kernel": int(v[0]), "cw": int(v[1]), "niss": int(v[2]),
                "source": ("default", "autotuned", "cache", "set")[v[3]], "candidates": cand}

    def stats(self):
        """Tree and list sizes (fmm_plan_stats); learned_p plans add the
        number of M2L pairs per order."""
        import numpy as np
        v = np.zeros(19, dtype=np.int64)
        self._c(lib().fmm_plan_stats(self.h, v.ctypes.data, 19))
        keys = ("cells", "leaves", "m2l_pairs", "p2p_pairs", "m2l_targets", "m2l_blocks_per_sm", "levels",
                "graph")
        out = dict(zip(keys, v[:8].tolist()))
        if self.cfg.learned_p:
            out["pairs_per_order"] = v[8:8 + self.cfg.p + 1].tolist()
        return out

    def pairs(self):
        """M2L pairs (target, source) as numpy int32 arrays, grouped by target."""
        import numpy as np
        cnt = ctypes.c_int64(0)
        self._c(lib().fmm_plan_pairs(self.h, None, None, 0, ctypes.byref(cnt)))
        t = np.zeros(cnt.value, dtype=np.int32)
        s = np.zeros(cnt.value, dtype=np.int32)
        self._c(lib().fmm_plan_pairs(self.h, t.ctypes.data, s.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return t, s

    def pair_data(self, labels=False, stream=None):
        """Device tensors: features [npair, 12] (float32) and, on request,
        labels [npair, 9] (float64) of the plan's M2L pairs."""
        t, _ = self.pairs()
        n = len(t)
        dev = torch.device("cuda", torch.cuda.current_device())
        feat = torch.empty((n, MLP_NF), dtype=torch.float32, device=dev)
        lab = torch.empty((n, MLP_NOUT), dtype=torch.float64, device=dev) if labels else None
        self._c(lib().fmm_pair_data(self.h, _ptr(feat), _ptr(lab), _stream(stream)))
        return feat, lab

    def set_mlp(self, blob):
        b = _host_f32(blob)
        self._c(lib().fmm_set_mlp(self.h, b.ctypes.data, len(b)))

    def pair_orders(self):
        """Order each M2L pair used in the last M2L (numpy int8, fmm_plan_pairs order)."""
        import numpy as np
        cnt = ctypes.c_int64(0)
        self._c(lib().fmm_plan_pair_orders(self.h, None, 0, ctypes.byref(cnt)))
        o = np.zeros(cnt.value, dtype=np.int8)
        self._c(lib().fmm_plan_pair_orders(self.h, o.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return o

    def set_pair_orders(self, orders):
        import numpy as np
        if orders is None:
            self._c(lib().fmm_set_pair_orders(self.h, None, 0))
            return
        o = np.ascontiguousarray(orders, dtype=np.int8)
        self._c(lib().fmm_set_pair_orders(self.h, o.ctypes.data, len(o)))

    def evaluate(self, x, y, z, q, stream=None):
        """Convenience: allocates outputs, returns (pot, acc[3, n]) device tensors."""
        n = len(x)
        out = torch.empty((4, n), dtype=torch.float64, device=x.device)
        self.fmm_evaluate(x, y, z, q, out[0], out[1], out[2], out[3], stream)
        return out[0], out[1:]
