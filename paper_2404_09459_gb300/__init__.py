"""GB300 randomized generalized singular values (arXiv:2404.09459).

Thin ctypes binding over the C ABI of `libgsvdrand.so` (include/gsvd_rand.h):
argument marshalling only; every step runs in the library's CUDA kernels.
PyTorch, when present, only supplies device memory and the current stream.
The library must be built first (`paper_2404_09459_gb300._build.build()`);
nothing here falls back to a CPU implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from ._build import LIB

__all__ = ["Context", "GsvdRandError", "load_library", "metrics_noalloc", "PREC", "LIB", "NOALLOC_MAX_N"]

PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "tf32x3": 3, "fp32": 4}
ERRORS = {-1: "ARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "BREAKDOWN", -6: "TOL_MISS",
          -7: "TIMEOUT", -8: "UNSUPPORTED", -9: "TOO_LARGE"}
FLAG_CHOL_FP64 = 1

EXPORTS = ("gsvd_rand_config_init", "gsvd_rand_create", "gsvd_rand_destroy", "gsvd_rand_last_error",
           "gsvd_rand_solve", "gsvd_rand_metrics", "gsvd_rand_gaussian", "gsvd_rand_philox",
           "gsvd_rand_profile_get", "gsvd_rand_profile_reset", "gsvd_rand_launch_count",
           "gsvd_rand_metrics_noalloc", "gsvd_rand_basis_cols", "gsvd_rand_solve_batched",
           "gsvd_rand_probe_features", "gsvd_rand_mlp_forward", "gsvd_rand_mlp_loss_grad", "gsvd_rand_mlp_adam",
           "gsvd_rand_mlp_train", "gsvd_rand_mlp_set", "gsvd_rand_mlp_load", "gsvd_rand_last_plan",
           "gsvd_rand_solve_grouped", "gsvd_rand_grouped_info", "gsvd_rand_chol64_retries",
           "gsvd_rand_product_shapes", "gsvd_rand_factors", "gsvd_rand_solve_complex", "gsvd_rand_grouped_basis_cols",
           "gsvd_rand_grouped_plans", "gsvd_rand_mlp_plan", "gsvd_rand_grouped_features")
NOALLOC_MAX_N = 32768
FLAG_PROFILE = 2
FLAG_BF16_SPLIT_POWER = 4
FLAG_BASIS_ONLY = 8
FLAG_ACC_RESID = 16
MLP_IN, MLP_HID, MLP_KCLS, MLP_QCLS, MLP_KBUCKET = 64, 128, 32, 5, 4
MLP_PARAMS = 64 * 128 + 128 + 128 * 128 + 128 + 128 * 37 + 37
STAGES = ("sketch", "gtq", "orth", "small", "small_gram", "small_jacobi", "small_refine", "small_cs", "setup",
          "proposal")


class GsvdRandError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gsvd_rand error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code
        self.name = ERRORS.get(code, "?")


class _Pair(C.Structure):
    _fields_ = [("G1", C.c_void_p), ("m", C.c_int64), ("ld1", C.c_int64), ("G2", C.c_void_p), ("p", C.c_int64),
                ("ld2", C.c_int64), ("n", C.c_int64), ("k", C.c_int), ("oversample", C.c_int), ("q", C.c_int),
                ("seed", C.c_uint64), ("pair", C.c_uint32), ("alpha", C.c_void_p), ("beta", C.c_void_p),
                ("r_out", C.c_void_p), ("resid_out", C.c_void_p), ("status", C.c_int)]


class _Config(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("prec", C.c_int), ("adaptive", C.c_int),
                ("block_b", C.c_int), ("tol", C.c_double), ("use_learned", C.c_int),
                ("mlp_path", C.c_char_p), ("flags", C.c_int)]


_lib = None


def load_library(path: str | None = None):
    """Load libgsvdrand.so (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_2404_09459_gb300._build.build()")
    lib = C.CDLL(path)
    vp, i64, i32, u64, u32 = C.c_void_p, C.c_int64, C.c_int, C.c_uint64, C.c_uint32
    dp = C.POINTER(C.c_double)
    lib.gsvd_rand_config_init.argtypes = [C.POINTER(_Config)]
    lib.gsvd_rand_create.argtypes = [C.POINTER(vp), C.POINTER(_Config)]
    lib.gsvd_rand_destroy.argtypes = [vp]
    lib.gsvd_rand_last_error.argtypes = [vp]
    lib.gsvd_rand_last_error.restype = C.c_char_p
    lib.gsvd_rand_solve.argtypes = [vp, vp, i64, i64, vp, i64, i64, i64, i32, i32, i32, u64, vp, vp, vp, vp]
    lib.gsvd_rand_grouped_basis_cols.argtypes = [vp, vp, i32]
    lib.gsvd_rand_grouped_plans.argtypes = [vp, vp, i32]
    lib.gsvd_rand_grouped_features.argtypes = [vp, vp, i32]
    lib.gsvd_rand_mlp_plan.argtypes = [vp, vp, i32, C.c_double, vp]
    lib.gsvd_rand_solve_complex.argtypes = [vp, vp, i64, i64, vp, i64, i64, i64, i32, i32, i32, u64, vp, vp, vp, vp]
    lib.gsvd_rand_metrics.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
    lib.gsvd_rand_gaussian.argtypes = [vp, i64, i64, u64, u32, u32, u32, vp]
    lib.gsvd_rand_philox.argtypes = [vp, u64, u64, u32, u32, u32, vp]
    lib.gsvd_rand_profile_get.argtypes = [vp, i32, dp, C.POINTER(C.c_int64)]
    lib.gsvd_rand_profile_reset.argtypes = [vp]
    lib.gsvd_rand_launch_count.argtypes = []
    lib.gsvd_rand_launch_count.restype = C.c_uint64
    lib.gsvd_rand_metrics_noalloc.argtypes = [i32, vp, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
    lib.gsvd_rand_basis_cols.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.gsvd_rand_solve_batched.argtypes = [vp, i32, C.POINTER(_Pair), i32]
    lib.gsvd_rand_solve_grouped.argtypes = [vp, i32, C.POINTER(_Pair)]
    lib.gsvd_rand_grouped_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                           C.POINTER(C.c_int64)]
    f32 = C.c_float
    lib.gsvd_rand_probe_features.argtypes = [vp, vp, i64, i64, vp, i64, i64, i64, u64, vp]
    lib.gsvd_rand_mlp_forward.argtypes = [vp, vp, vp, vp, i32, i32, vp]
    lib.gsvd_rand_mlp_loss_grad.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp, vp]
    lib.gsvd_rand_mlp_adam.argtypes = [vp, vp, vp, vp, vp, i32, f32, f32, f32, f32]
    lib.gsvd_rand_mlp_train.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, f32, vp]
    lib.gsvd_rand_mlp_set.argtypes = [vp, vp, vp]
    lib.gsvd_rand_mlp_load.argtypes = [vp, C.c_char_p]
    lib.gsvd_rand_last_plan.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.gsvd_rand_chol64_retries.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.gsvd_rand_product_shapes.argtypes = [vp, C.POINTER(C.c_int)]
    lib.gsvd_rand_factors.argtypes = [vp, vp, i64, vp, i64, vp, i64]
    for name in EXPORTS:
        if name not in ("gsvd_rand_last_error", "gsvd_rand_launch_count"):
            getattr(lib, name).restype = C.c_int
    if path == LIB:
        _lib = lib
    return lib


def _cmat_ptr(x, want_dtype: str):
    """(pointer, rows, cols, ld in complex entries, on_device, keepalive) of a row-major complex
    matrix: complex128 for "c128", complex64 for "c64" (interleaved (re, im) pairs)."""
    if _is_torch(x):
        import torch
        dt = {"c128": torch.complex128, "c64": torch.complex64}[want_dtype]
        if x.dtype != dt:
            raise TypeError(f"expected {dt}, got {x.dtype}")
        if x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("matrix must be 2-D with unit column stride (row-major)")
        return x.data_ptr(), x.shape[0], x.shape[1], max(x.stride(0), x.shape[1]), x.is_cuda, x
    import numpy as np
    dt = {"c128": np.complex128, "c64": np.complex64}[want_dtype]
    a = np.asarray(x)
    if a.dtype != dt:
        raise TypeError(f"expected {np.dtype(dt)}, got {a.dtype}")
    if a.ndim != 2 or a.strides[1] != a.itemsize or a.strides[0] % a.itemsize:
        raise ValueError("matrix must be 2-D row-major")
    return a.ctypes.data, a.shape[0], a.shape[1], max(a.strides[0] // a.itemsize, a.shape[1]), False, a


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _mat_ptr(x, want_dtype: str):
    """(pointer, rows, cols, ld, on_device, keepalive) of a row-major matrix."""
    if _is_torch(x):
        import torch
        dt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[want_dtype]
        if x.dtype != dt:
            raise TypeError(f"expected {dt}, got {x.dtype}")
        if x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("matrix must be 2-D with unit column stride (row-major)")
        return x.data_ptr(), x.shape[0], x.shape[1], max(x.stride(0), x.shape[1]), x.is_cuda, x
    import numpy as np
    dt = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16}[want_dtype]  # bf16: raw bit patterns
    a = np.asarray(x)
    if a.dtype != dt:
        raise TypeError(f"expected {np.dtype(dt)}, got {a.dtype}")
    if a.ndim != 2 or a.strides[1] != a.itemsize or a.strides[0] % a.itemsize:
        raise ValueError("matrix must be 2-D row-major")
    return a.ctypes.data, a.shape[0], a.shape[1], max(a.strides[0] // a.itemsize, a.shape[1]), False, a


class Context:
    """One library context (device, stream, precision).

    prec: "fp64" | "tf32" | "tf32x3" | "bf16" | "fp32".  stream: a torch.cuda.Stream,
    a raw cudaStream_t int, or None for torch's current stream (legacy default
    stream without torch).
    """

    def __init__(self, prec: str = "tf32", device: int = 0, stream=None, flags: int = 0,
                 adaptive: bool = False, block_b: int = 100, tol: float = 1e-4, use_learned: bool = False,
                 mlp_path: str | None = None):
        self.lib = load_library()
        cfg = _Config()
        self.lib.gsvd_rand_config_init(C.byref(cfg))
        cfg.device = device
        cfg.prec = PREC[prec]
        cfg.flags = flags
        cfg.adaptive = 1 if adaptive else 0
        cfg.block_b = block_b
        cfg.tol = tol
        cfg.use_learned = 1 if use_learned else 0
        self._learned = bool(use_learned)
        self._mlp_path = mlp_path.encode() if mlp_path else None
        cfg.mlp_path = self._mlp_path
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device)
            except ImportError:
                stream = None
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        cfg.stream = C.c_void_p(int(stream) if stream else 0)
        self.prec = prec
        self.device = device
        self._stream = stream
        h = C.c_void_p()
        rc = self.lib.gsvd_rand_create(C.byref(h), C.byref(cfg))
        if rc:
            raise GsvdRandError(rc, "create failed")
        self.h = h

    # ------------------------------------------------------------------ util
    def _check(self, rc):
        if rc:
            raise GsvdRandError(rc, self.lib.gsvd_rand_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gsvd_rand_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _out_vec(self, on_device: bool, n: int, dtype="f64"):
        if on_device:
            import torch
            dt = {"f64": torch.float64, "u32": torch.int32}[dtype]
            t = torch.empty(n, dtype=dt, device=f"cuda:{self.device}")
            return t, t.data_ptr()
        import numpy as np
        a = np.empty(n, dtype={"f64": np.float64, "u32": np.uint32}[dtype])
        return a, a.ctypes.data

    # ------------------------------------------------------------------ API
    def _g_dtype(self):
        return {"fp64": "f64", "bf16": "bf16"}.get(self.prec, "f32")

    def solve(self, G1, G2, k: int, oversample: int = 10, q: int = 1, seed: int = 0):
        """Randomized GSVs of {G1, G2}: dict(alpha, beta, r, resid).

        Outputs live where G1 lives (CUDA tensors for CUDA inputs, numpy otherwise)."""
        want = self._g_dtype()
        p1, m, n1, ld1, dev1, k1 = _mat_ptr(G1, want)
        p2, p, n2, ld2, dev2, k2 = _mat_ptr(G2, want)
        if n1 != n2:
            raise ValueError("G1 and G2 must have the same number of columns")
        alpha, pa = self._out_vec(dev1, k)
        beta, pb = self._out_vec(dev1, k)
        r = C.c_int(0)
        resid = (C.c_double * 2)()
        rc = self.lib.gsvd_rand_solve(self.h, p1, m, ld1, p2, p, ld2, n1, k, oversample, q, seed, pa, pb,
                                      C.addressof(r), C.addressof(resid))
        self._check(rc)
        rr = r.value
        self._last_shape = (m, p, n1, rr)
        return dict(alpha=alpha[:rr], beta=beta[:rr], r=rr, resid=(resid[0], resid[1]))

    def solve_complex(self, G1, G2, k: int, oversample: int = 10, q: int = 1, seed: int = 0):
        """Randomized GSVs of a complex pair (gsvd_rand_solve_complex): complex128 matrices on
        the FP64 path, complex64 otherwise.  dict(alpha, beta, r, resid); outputs live where G1
        lives."""
        want = "c128" if self.prec == "fp64" else "c64"
        p1, m, n1, ld1, dev1, k1 = _cmat_ptr(G1, want)
        p2, p, n2, ld2, dev2, k2 = _cmat_ptr(G2, want)
        if n1 != n2:
            raise ValueError("G1 and G2 must have the same number of columns")
        alpha, pa = self._out_vec(dev1, k)
        beta, pb = self._out_vec(dev1, k)
        r = C.c_int(0)
        resid = (C.c_double * 2)()
        rc = self.lib.gsvd_rand_solve_complex(self.h, p1, m, ld1, p2, p, ld2, n1, k, oversample, q, seed, pa, pb,
                                              C.addressof(r), C.addressof(resid))
        self._check(rc)
        return dict(alpha=alpha[:r.value], beta=beta[:r.value], r=r.value, resid=(resid[0], resid[1]))

    def factors(self):
        """GSVD factors of the last solve(): dict(U (m x r), V (p x r), R (r x n)), FP64 CUDA tensors,
        with G1 ~ U diag(alpha) R and G2 ~ V diag(beta) R (gsvd_rand_factors)."""
        import torch
        m, p, n, r = getattr(self, "_last_shape", (0, 0, 0, 0))
        dev = torch.device("cuda", self.device)
        U = torch.empty((m, r), dtype=torch.float64, device=dev)
        V = torch.empty((p, r), dtype=torch.float64, device=dev)
        R = torch.empty((r, n), dtype=torch.float64, device=dev)
        self._check(self.lib.gsvd_rand_factors(self.h, U.data_ptr() if U.numel() else None, max(r, 1),
                                               V.data_ptr() if V.numel() else None, max(r, 1),
                                               R.data_ptr() if R.numel() else None, max(n, 1)))
        return dict(U=U, V=V, R=R)

    def solve_batched(self, pairs, workers: int = 8):
        """Many independent pairs at once.  pairs: sequence of dicts with G1, G2, k and optional
        oversample (10), q (1), seed (0), pair (its index).  Returns a list of dict(alpha, beta, r,
        resid, status); raises GsvdRandError if any pair failed (after all ran)."""
        return self._many(pairs, workers)

    def solve_grouped(self, pairs, host_out: bool = False):
        """The same as solve_batched, as one grouped solve: every step one launch for all pairs,
        the sequence captured into a CUDA graph and replayed while the inputs stay the same.
        host_out: alpha / beta returned in host memory (numpy) even for device inputs."""
        return self._many(pairs, None, host_out)

    def grouped_plans(self, npairs: int):
        """[(k, q, fallback)] per pair of the last learned grouped solve."""
        c = (C.c_int * (3 * npairs))()
        self._check(self.lib.gsvd_rand_grouped_plans(self.h, c, npairs))
        return [(c[3 * i], c[3 * i + 1], c[3 * i + 2]) for i in range(npairs)]

    def grouped_features(self, npairs: int):
        """(npairs, 64) float32 probe features of the last learned grouped solve."""
        import numpy as np
        f = np.zeros((npairs, MLP_IN), np.float32)
        self._check(self.lib.gsvd_rand_grouped_features(self.h, f.ctypes.data, npairs))
        return f

    def grouped_basis_cols(self, npairs: int):
        """[(l1, l2)] per pair of the last grouped adaptive solve (Algorithm 1 basis columns)."""
        c = (C.c_int * (2 * npairs))()
        self._check(self.lib.gsvd_rand_grouped_basis_cols(self.h, c, npairs))
        return [(c[2 * i], c[2 * i + 1]) for i in range(npairs)]

    def grouped_info(self):
        """dict(tuned=[(stages, ctas_per_sm)] x 3 (first sketch, power sketch, G^T Q), captures,
        replays, launches per replay) of the last grouped plan."""
        t = (C.c_int * 6)()
        c, r, n = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        self._check(self.lib.gsvd_rand_grouped_info(self.h, t, C.byref(c), C.byref(r), C.byref(n)))
        return dict(tuned=[(t[0], t[1]), (t[2], t[3]), (t[4], t[5])], captures=c.value, replays=r.value,
                    launches=n.value)

    def _many(self, pairs, workers, host_out=False):
        want = self._g_dtype()
        arr = (_Pair * len(pairs))()
        outs, keep = [], []
        for i, d in enumerate(pairs):
            p1, m, n1, ld1, dev1, k1 = _mat_ptr(d["G1"], want)
            p2, p, n2, ld2, dev2, k2 = _mat_ptr(d["G2"], want)
            if n1 != n2:
                raise ValueError(f"pair {i}: G1 and G2 must have the same number of columns")
            k = int(d["k"])
            alpha, pa = self._out_vec(dev1 and not host_out, k)
            beta, pb = self._out_vec(dev1 and not host_out, k)
            r = C.c_int(0)
            resid = (C.c_double * 2)()
            q = arr[i]
            q.G1, q.m, q.ld1, q.G2, q.p, q.ld2, q.n = p1, m, ld1, p2, p, ld2, n1
            q.k, q.oversample, q.q = k, int(d.get("oversample", 10)), int(d.get("q", 1))
            q.seed, q.pair = int(d.get("seed", 0)), int(d.get("pair", i))
            q.alpha, q.beta, q.r_out, q.resid_out = pa, pb, C.addressof(r), C.addressof(resid)
            outs.append((alpha, beta, r, resid))
            keep += [k1, k2]
        if workers is None:
            rc = self.lib.gsvd_rand_solve_grouped(self.h, len(pairs), arr)
        else:
            rc = self.lib.gsvd_rand_solve_batched(self.h, len(pairs), arr, workers)
        res = [dict(alpha=a[:r.value], beta=b[:r.value], r=r.value, resid=(rs[0], rs[1]), status=arr[i].status)
               for i, (a, b, r, rs) in enumerate(outs)]
        del keep
        self._check(rc)
        return res

    # ------------------------------------------------------------------ learned proposal
    def probe_features(self, G1, G2, seed: int = 0):
        """The 64 probe features (float32; a CUDA tensor for CUDA inputs, numpy otherwise)."""
        want = self._g_dtype()
        p1, m, n1, ld1, dev1, k1 = _mat_ptr(G1, want)
        p2, p, n2, ld2, dev2, k2 = _mat_ptr(G2, want)
        if n1 != n2:
            raise ValueError("G1 and G2 must have the same number of columns")
        if dev1:
            import torch
            out = torch.empty(MLP_IN, dtype=torch.float32, device=f"cuda:{self.device}")
            ptr = out.data_ptr()
        else:
            import numpy as np
            out = np.empty(MLP_IN, dtype=np.float32)
            ptr = out.ctypes.data
        self._check(self.lib.gsvd_rand_probe_features(self.h, p1, m, ld1, p2, p, ld2, n1, seed, ptr))
        return out

    @staticmethod
    def _dev_ptr(t, dtype, numel=None):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
        if numel is not None and t.numel() < numel:
            raise ValueError(f"tensor holds {t.numel()} elements, {numel} needed")
        return t.data_ptr()

    def mlp_forward(self, params, norm, X, bf16: bool = False):
        """Logits (B x 37) of X (B x 64); all CUDA float32 tensors."""
        import torch
        B = X.shape[0]
        z = torch.empty(B, MLP_KCLS + MLP_QCLS, dtype=torch.float32, device=X.device)
        f = torch.float32
        self._check(self.lib.gsvd_rand_mlp_forward(self.h, self._dev_ptr(params, f, MLP_PARAMS),
                                                   self._dev_ptr(norm, f, 2 * MLP_IN), self._dev_ptr(X, f, B * MLP_IN),
                                                   B, 1 if bf16 else 0, z.data_ptr()))
        return z

    def mlp_loss_grad(self, params, norm, X, yk, yq):
        """(loss, grad) of the batch; labels int32 CUDA tensors."""
        import torch
        B = X.shape[0]
        f, i = torch.float32, torch.int32
        grad = torch.empty(MLP_PARAMS, dtype=f, device=X.device)
        loss = torch.empty(1, dtype=f, device=X.device)
        self._check(self.lib.gsvd_rand_mlp_loss_grad(self.h, self._dev_ptr(params, f, MLP_PARAMS),
                                                     self._dev_ptr(norm, f, 2 * MLP_IN),
                                                     self._dev_ptr(X, f, B * MLP_IN), self._dev_ptr(yk, i, B),
                                                     self._dev_ptr(yq, i, B), B, grad.data_ptr(), loss.data_ptr()))
        return float(loss.item()), grad

    def mlp_adam(self, params, m, v, grad, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        import torch
        f = torch.float32
        self._check(self.lib.gsvd_rand_mlp_adam(self.h, self._dev_ptr(params, f, MLP_PARAMS),
                                                self._dev_ptr(m, f, MLP_PARAMS), self._dev_ptr(v, f, MLP_PARAMS),
                                                self._dev_ptr(grad, f, MLP_PARAMS), t, lr, beta1, beta2, eps))

    def mlp_train(self, params, m, v, norm, X, yk, yq, order, B: int, t0: int, lr: float):
        """len(order) // B Adam steps over the row indices `order` (int32 CUDA); returns the
        per-step losses (CUDA float32)."""
        import torch
        f, i = torch.float32, torch.int32
        N = X.shape[0]
        steps = order.numel() // B
        hist = torch.empty(max(steps, 1), dtype=f, device=X.device)
        self._check(self.lib.gsvd_rand_mlp_train(
            self.h, self._dev_ptr(params, f, MLP_PARAMS), self._dev_ptr(m, f, MLP_PARAMS),
            self._dev_ptr(v, f, MLP_PARAMS), self._dev_ptr(norm, f, 2 * MLP_IN), self._dev_ptr(X, f, N * MLP_IN),
            self._dev_ptr(yk, i, N), self._dev_ptr(yq, i, N), self._dev_ptr(order, i, steps * B), steps, B, t0,
            lr, hist.data_ptr()))
        return hist[:steps]

    def mlp_plan(self, logits, quantile: float = 0.9):
        """(k, q, k bucket) per row of device logits (B x 37), the learned solve's rule on the device."""
        import numpy as np
        B = int(logits.shape[0])
        out = np.zeros(3 * B, np.int32)
        self._check(self.lib.gsvd_rand_mlp_plan(self.h, logits.data_ptr(), B, float(quantile), out.ctypes.data))
        return out.reshape(B, 3)

    def mlp_set(self, params, norm):
        """The network of the learned solve (float32, CUDA tensors or numpy)."""
        import numpy as np
        keep = []

        def ptr(a):
            if _is_torch(a):
                a = a.contiguous()
                keep.append(a)
                return a.data_ptr()
            a = np.ascontiguousarray(a, dtype=np.float32)
            keep.append(a)
            return a.ctypes.data
        self._check(self.lib.gsvd_rand_mlp_set(self.h, ptr(params), ptr(norm)))

    def mlp_load(self, path: str):
        self._check(self.lib.gsvd_rand_mlp_load(self.h, path.encode()))

    def last_plan(self):
        """(k, q, fallback) of the last learned solve."""
        k, q, fb = C.c_int(0), C.c_int(0), C.c_int(0)
        self._check(self.lib.gsvd_rand_last_plan(self.h, C.byref(k), C.byref(q), C.byref(fb)))
        return k.value, q.value, bool(fb.value)

    def basis_cols(self):
        """Columns (l1, l2) of the two bases of the last solve."""
        a, b = C.c_int(0), C.c_int(0)
        self._check(self.lib.gsvd_rand_basis_cols(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def product_shapes(self):
        """[(stages, ctas_per_sm)] x 3 (first sketch, power sketch, G^T Q) of the last solve whose
        two-side products ran as grouped launches, as the built-in tuner picked them."""
        t = (C.c_int * 6)()
        self._check(self.lib.gsvd_rand_product_shapes(self.h, t))
        return [(t[0], t[1]), (t[2], t[3]), (t[4], t[5])]

    def chol64_retries(self) -> int:
        """Solves (on this context and its batched workers) repeated with FP64 Cholesky
        factors after their FP32 CholeskyQR broke down."""
        c = C.c_int64(0)
        self._check(self.lib.gsvd_rand_chol64_retries(self.h, C.byref(c)))
        return c.value

    def metrics(self, alpha, beta, pad_to_n: int = 0, pad_mode: int = 0):
        """Section 1 quantities: dict(theta, rho, P1, P2, D1, D2)."""
        import numpy as np
        on_dev = _is_torch(alpha) and alpha.is_cuda
        if _is_torch(alpha):
            pa, pb, r = alpha.data_ptr(), beta.data_ptr(), alpha.numel()
            keep = (alpha, beta)
        else:
            a = np.ascontiguousarray(alpha, dtype=np.float64)
            b = np.ascontiguousarray(beta, dtype=np.float64)
            pa, pb, r = a.ctypes.data, b.ctypes.data, a.size
            keep = (a, b)
        N = max(pad_to_n, r)
        outs = [self._out_vec(on_dev, N) for _ in range(4)]
        D, pD = self._out_vec(on_dev, 2)
        rc = self.lib.gsvd_rand_metrics(self.h, pa, pb, r, pad_to_n, pad_mode, *[o[1] for o in outs], pD)
        del keep
        self._check(rc)
        return dict(theta=outs[0][0], rho=outs[1][0], P1=outs[2][0], P2=outs[3][0], D1=D[0], D2=D[1])

    def gaussian(self, n: int, l: int, seed: int, pair: int = 0, side: int = 0, stream: int = 0,
                 device_out: bool = False):
        """The n x l Gaussian test matrix (FP64) the solver draws."""
        out, ptr = self._out_vec(device_out, n * l)
        self._check(self.lib.gsvd_rand_gaussian(self.h, n, l, seed, pair, side, stream, ptr))
        return out.reshape(n, l)

    def profile(self, reset: bool = False):
        """Per-stage device time (ms) and call counts recorded under FLAG_PROFILE."""
        out = {}
        for i, name in enumerate(STAGES):
            ms = C.c_double()
            n = C.c_int64()
            self._check(self.lib.gsvd_rand_profile_get(self.h, i, C.byref(ms), C.byref(n)))
            out[name] = (ms.value, n.value)
        if reset:
            self.lib.gsvd_rand_profile_reset(self.h)
        return out

    def launch_count(self) -> int:
        """Kernels launched by the library so far in this process."""
        return int(self.lib.gsvd_rand_launch_count())

    def philox(self, count: int, seed: int, pair: int = 0, side: int = 0, stream: int = 0):
        """Raw Philox4x32-10 words, shape (count, 4) uint32 (host)."""
        out, ptr = self._out_vec(False, 4 * count, "u32")
        self._check(self.lib.gsvd_rand_philox(self.h, count, seed, pair, side, stream, ptr))
        return out.reshape(count, 4)


def metrics_noalloc(alpha, beta, pad_to_n: int = 0, pad_mode: int = 0, device: int = 0, stream=None, out=None):
    """Context.metrics through gsvd_rand_metrics_noalloc, for callers that must not
    allocate device memory: the library uses a fixed static scratch instead.

    numpy inputs give numpy outputs (host memory only).  CUDA tensor inputs need
    `out`, a dict of caller-owned CUDA float64 tensors theta, rho, P1, P2 (N each)
    and D (2), which is filled and returned; nothing is allocated on the device.
    stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (legacy default
    stream).  N = max(len(alpha), pad_to_n) must not exceed NOALLOC_MAX_N.
    Calls that overlap in time share the scratch and race."""
    import numpy as np
    lib = load_library()
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    sp = C.c_void_p(int(stream) if stream else 0)
    if _is_torch(alpha) and alpha.is_cuda:
        if out is None:
            raise ValueError("CUDA inputs need caller-owned outputs: out=dict(theta, rho, P1, P2, D)")
        pa, pb, r = alpha.data_ptr(), beta.data_ptr(), alpha.numel()
        N = max(pad_to_n, r)
        for key, size in (("theta", N), ("rho", N), ("P1", N), ("P2", N), ("D", 2)):
            t = out[key]
            if not (t.is_cuda and t.dtype == alpha.dtype and t.numel() >= size and t.is_contiguous()):
                raise ValueError(f"out[{key!r}] must be a contiguous CUDA float64 tensor of >= {size} elements")
        ptrs = [out[k].data_ptr() for k in ("theta", "rho", "P1", "P2", "D")]
        res = out
    else:
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        b = np.ascontiguousarray(beta, dtype=np.float64)
        pa, pb, r = a.ctypes.data, b.ctypes.data, a.size
        N = max(pad_to_n, r)
        res = {k: np.empty(N if k != "D" else 2) for k in ("theta", "rho", "P1", "P2", "D")}
        ptrs = [res[k].ctypes.data for k in ("theta", "rho", "P1", "P2", "D")]
    rc = lib.gsvd_rand_metrics_noalloc(device, sp, pa, pb, r, pad_to_n, pad_mode, *ptrs)
    if rc:
        why = (f"N = {N} pairs exceeds the fixed limit {NOALLOC_MAX_N}" if rc == -9
               else "bad arguments or CUDA failure")
        raise GsvdRandError(rc, why)
    return dict(theta=res["theta"], rho=res["rho"], P1=res["P1"], P2=res["P2"], D1=res["D"][0], D2=res["D"][1])
