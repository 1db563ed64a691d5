"""Python binding of libpsdproj (include/psdproj.h): randomized PSD-cone
projections (arXiv 2410.19208, Algs. 1-5) on one GB300 GPU.

This module only marshals arguments: every step runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU path:
if the compiled library is missing, importing the binding raises.

Layouts (same as the C ABI):
* A, P: square FP32 tensors, row-major (stride(1) == 1), only the upper
  triangle of A is read.
* tall matrices (Omega, Y, Q, W): shape (n, m) COLUMN-major, i.e. stride(0)
  == 1 and stride(1) = ld >= n.  ``tall_empty(n, m)`` makes one.
* small matrices (core C, V): shape (m, m) column-major (use ``.t()`` of a
  row-major tensor).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpsdproj.so")

PREC_FP32, PREC_TF32, PREC_BF16, PREC_BF16X3 = 0, 1, 2, 3
OUT_FULL, OUT_UPPER, OUT_FACTOR = 0, 1, 2
EIG_AUTO, EIG_JACOBI, EIG_TRIDIAG = 0, 1, 2
SKETCH_GAUSS, SKETCH_SRHT = 0, 1
ALPHA_MINEIG, ALPHA_RITZ = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTFINITE", 4: "ENOCONV", 5: "ETIMEOUT",
          6: "ECUDA", 7: "ENOTSUP", 8: "ETOOLARGE"}


class PsdprojError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("syrk_prec", ctypes.c_int), ("N", ctypes.c_int),
                ("out_mode", ctypes.c_int), ("eig", ctypes.c_int), ("sketch", ctypes.c_int),
                ("alpha_mode", ctypes.c_int), ("deterministic", ctypes.c_int), ("spin_limit", ctypes.c_int64),
                ("reserved", ctypes.c_int * 2)]


class Problem(ctypes.Structure):
    """psdproj_problem: one projection of a psdproj_batched call."""
    _fields_ = [("dA", ctypes.c_void_p), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("k", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("algorithm", ctypes.c_int), ("seed", ctypes.c_uint64), ("alpha_in", ctypes.c_double),
                ("d_alpha_out", ctypes.c_void_p), ("d_info", ctypes.c_void_p),
                ("dP", ctypes.c_void_p), ("ldp", ctypes.c_int64),
                ("dW", ctypes.c_void_p), ("ldw", ctypes.c_int64), ("d_rank", ctypes.c_void_p)]


class Request(ctypes.Structure):
    """psdproj_request: one request to a psdproj_server."""
    _fields_ = Problem._fields_ + [("footprint_bytes", ctypes.c_int64)]


class Sdls(ctypes.Structure):
    """psdproj_sdls: the semidefinite least-squares problem of Alg. 6."""
    _fields_ = [("dC", ctypes.c_void_p), ("dA", ctypes.POINTER(ctypes.c_void_p)), ("b", ctypes.POINTER(ctypes.c_double)),
                ("n", ctypes.c_int64), ("ld", ctypes.c_int64), ("rho", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps", ctypes.c_double), ("seed", ctypes.c_uint64), ("mc", ctypes.c_int), ("k", ctypes.c_int),
                ("p", ctypes.c_int), ("q", ctypes.c_int), ("algorithm", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("reserved", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    """psdproj_server_stats."""
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("inflight_bytes", ctypes.c_int64),
                ("inflight_peak_bytes", ctypes.c_int64), ("admit_bytes", ctypes.c_int64),
                ("last_error_status", ctypes.c_int), ("last_error_cuda", ctypes.c_int),
                ("last_error_line", ctypes.c_int), ("reserved", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_u64 = ctypes.c_uint64


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpsdproj.so not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "psdproj_default_opts": (None, [ctypes.POINTER(Opts)]),
        "psdproj_create": (_int, [ctypes.POINTER(_P), _int, _P, ctypes.c_size_t]),
        "psdproj_set_stream": (_int, [_P, _P]),
        "psdproj_destroy": (_int, [_P]),
        "psdproj_sync_status": (_int, [_P]),
        "psdproj_status_string": (ctypes.c_char_p, [_int]),
        "psdproj_workspace_bytes": (ctypes.c_size_t, [_P]),
        "psdproj_projection_bytes": (ctypes.c_size_t, [_i64, _int, _int, ctypes.POINTER(Opts)]),
        "psdproj_alg1": (_int, [_P, _P, _i64, _i64, _int, _int, _int, _u64, _P, _i64, _P, _i64,
                                _P, ctypes.POINTER(Opts)]),
        "psdproj_batched": (_int, [_P, _int, _P, _P]),
        "psdproj_batched_graph": (_int, [_P, _int, _P, _P]),
        "psdproj_batched_grouped": (_int, [_P, _int, _P, _P]),
        "psdproj_set_batch_streams": (_int, [_P, _int]),
        "psdproj_tune_batch": (_int, [_P, _int, _P, _P, _int, ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_double)]),
        "psdproj_tune_lookup": (_int, [ctypes.c_char_p, _int, _i64, _int, ctypes.POINTER(_int)]),
        "psdproj_tune_store": (_int, [ctypes.c_char_p, _int, _i64, _int, _int]),
        "psdproj_set_reserved_sms": (_int, [_P, _int]),
        "psdproj_alg2": (_int, [_P, _P, _i64, _i64, _int, _int, _int, _u64, ctypes.c_double,
                                _P, _P, _P, _i64, _P, _i64, _P, ctypes.POINTER(Opts)]),
        "psdproj_alg1_host": (_int, [_P, _P, _i64, _i64, _int, _int, _int, _u64, _P, _i64, _P,
                                     _i64, _P, ctypes.POINTER(Opts)]),
        "psdproj_alg2_host": (_int, [_P, _P, _i64, _i64, _int, _int, _int, _u64,
                                     ctypes.c_double, _P, _P, _i64, _P, _i64, _P,
                                     ctypes.POINTER(Opts)]),
        "psdproj_gaussian": (_int, [_P, _u64, ctypes.c_uint32, _i64, _int, _P, _i64]),
        "psdproj_srht": (_int, [_P, _u64, _i64, _int, _P, _i64]),
        "psdproj_sym_pass": (_int, [_P, _P, _i64, _i64, _P, _i64, _int, _P, _P, _i64, _int]),
        "psdproj_cholqr2": (_int, [_P, _P, _i64, _i64, _int, _P, _i64, _P]),
        "psdproj_core": (_int, [_P, _P, _i64, _P, _i64, _i64, _int, _P]),
        "psdproj_eig": (_int, [_P, _P, _int, _P, _P]),
        "psdproj_eig_method": (_int, [_P, _P, _int, _P, _P, _int]),
        "psdproj_factor": (_int, [_P, _P, _i64, _i64, _int, _P, _P, _P, _i64, _P]),
        "psdproj_syrk": (_int, [_P, _P, _i64, _i64, _int, _P, _P, _i64, _int, _int]),
        "psdproj_min_eig": (_int, [_P, _P, _i64, _i64, _int, _u64, _P, _P, _P]),
        "psdproj_min_eig_noalloc": (_int, [_P, _i64, _i64, _int, _u64, _P, _P, _P, _P]),
        "psdproj_server_create": (_int, [ctypes.POINTER(_P), _int, _int, ctypes.c_size_t, ctypes.POINTER(Opts)]),
        "psdproj_server_submit": (_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(_u64)]),
        "psdproj_server_wait": (_int, [_P, _u64, ctypes.c_double, ctypes.POINTER(_int),
                                       ctypes.POINTER(ctypes.c_double)]),
        "psdproj_server_drain": (_int, [_P, ctypes.c_double]),
        "psdproj_server_get_stats": (_int, [_P, ctypes.POINTER(ServerStats)]),
        "psdproj_server_destroy": (_int, [_P]),
        "psdproj_last_cuda_error": (_int, [ctypes.POINTER(_int)]),
        "psdproj_sdls_dual_gd": (_int, [_P, ctypes.POINTER(Sdls), ctypes.POINTER(ctypes.c_double), _P, _i64,
                                        ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Opts)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def lib():
    return _load()


def _check(code: int, what: str):
    if code != 0:
        if code in (2, 6, 7):     # ENOMEM, ECUDA, ENOTSUP: name the CUDA error behind it
            line = _int(0)
            err = _load().psdproj_last_cuda_error(ctypes.byref(line))
            if err:
                what = f"{what} (cudaError {err} at C-ABI line {line.value})"
        raise PsdprojError(code, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _sq(A, name="A"):
    assert A.is_cuda and A.dtype == torch.float32 and A.dim() == 2, name
    assert A.shape[0] == A.shape[1] and A.stride(1) == 1, f"{name}: row-major square FP32"
    return A.shape[0], A.stride(0)


def _tall(X, name="X"):
    assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2, name
    assert X.stride(0) == 1 or X.shape[1] == 1, f"{name}: column-major (stride(0) == 1)"
    ld = X.stride(1) if X.shape[1] > 1 else max(X.shape[0], X.stride(1))
    return X.shape[0], X.shape[1], ld


def tall_empty(n: int, m: int, device="cuda", ld: int | None = None):
    """Column-major n x m FP32 device tensor (shape (n, m), stride (1, ld))."""
    ld = ld or n
    return torch.empty(m, ld, dtype=torch.float32, device=device).t()[:n]


def projection_bytes(n: int, k: int, p: int, opts: Opts | None = None) -> int:
    """Device bytes a context allocates for one projection (psdproj_projection_bytes)."""
    return int(_load().psdproj_projection_bytes(n, k, p, ctypes.byref(opts) if opts else None))


def make_opts(prec=PREC_FP32, syrk_prec=PREC_FP32, N=10, out_mode=OUT_FULL,
              eig=EIG_AUTO, sketch=SKETCH_GAUSS, alpha_mode=ALPHA_MINEIG, deterministic=0,
              spin_limit=0) -> Opts:
    o = Opts()
    _load().psdproj_default_opts(ctypes.byref(o))
    o.prec, o.syrk_prec, o.N, o.out_mode, o.eig = prec, syrk_prec, N, out_mode, eig
    o.sketch, o.alpha_mode = sketch, alpha_mode
    o.deterministic, o.spin_limit = int(deterministic), int(spin_limit)
    return o


class Context:
    """A psdproj context bound to one device and one CUDA stream; hbm_budget
    (bytes, 0 = no cap) caps the device memory it may hold."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, hbm_budget: int = 0):
        lib = _load()
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        _check(lib.psdproj_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                  int(hbm_budget)), "psdproj_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _load().psdproj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        _check(_load().psdproj_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "set_stream")

    def sync_status(self) -> int:
        return _load().psdproj_sync_status(self.h)

    def workspace_bytes(self) -> int:
        return int(_load().psdproj_workspace_bytes(self.h))

    # ---- whole projections ------------------------------------------------
    def alg1(self, A, k, p, q, seed, P=None, W=None, rank=None, opts: Opts | None = None):
        n, lda = _sq(A)
        ldp = P.stride(0) if P is not None else n
        ldw = _tall(W, "W")[2] if W is not None else n
        _check(_load().psdproj_alg1(self.h, _ptr(A), n, lda, k, p, q, seed, _ptr(P), ldp, _ptr(W),
                                    ldw, _ptr(rank), ctypes.byref(opts) if opts else None),
               "psdproj_alg1")

    def alg2(self, A, k, p, q, seed, alpha_in=0.0, alpha_out=None, info=None, P=None, W=None,
             rank=None, opts: Opts | None = None):
        n, lda = _sq(A)
        ldp = P.stride(0) if P is not None else n
        ldw = _tall(W, "W")[2] if W is not None else n
        _check(_load().psdproj_alg2(self.h, _ptr(A), n, lda, k, p, q, seed, float(alpha_in),
                                    _ptr(alpha_out), _ptr(info), _ptr(P), ldp, _ptr(W), ldw,
                                    _ptr(rank), ctypes.byref(opts) if opts else None),
               "psdproj_alg2")

    @staticmethod
    def _problem_table(problems):
        arr = (Problem * max(1, len(problems)))()
        for i, d in enumerate(problems):
            A = d["A"]
            n, lda = _sq(A)
            P, W = d.get("P"), d.get("W")
            arr[i] = Problem(_ptr(A), n, lda, d["k"], d["p"], d["q"], d.get("algorithm", 1), d["seed"],
                             float(d.get("alpha_in", 0.0)), _ptr(d.get("alpha_out")), _ptr(d.get("info")),
                             _ptr(P), P.stride(0) if P is not None else n,
                             _ptr(W), _tall(W, "W")[2] if W is not None else n, _ptr(d.get("rank")))
        return arr

    def batched(self, problems, opts: Opts | None = None, graph: bool = False, grouped: bool = False):
        """problems: list of dicts with keys A, k, p, q, seed, algorithm (1 or 2) and
        optional P, W, rank, alpha_in, alpha_out, info (device tensors).
        graph=True: psdproj_batched_graph (recorded once into a CUDA graph and
        replayed while the table is unchanged); grouped=True:
        psdproj_batched_grouped (the small steps as grouped launches, also
        recorded and replayed)."""
        arr = self._problem_table(problems)
        name = "psdproj_batched_grouped" if grouped else ("psdproj_batched_graph" if graph else "psdproj_batched")
        _check(getattr(_load(), name)(self.h, len(problems), ctypes.byref(arr),
                                      ctypes.byref(opts) if opts else None), name)

    def sdls(self, C, As, b, rho, k, p, q, algorithm, beta, eps, max_iter, seed, y0, warm_start=False,
             X=None, opts: Opts | None = None):
        """Alg. 6 on device matrices C, As (n x n, row-major, upper read) and host b.
        Returns dict(y, iters, gnorm, hist)."""
        n, ld = _sq(C, "C")
        for A in As:
            assert _sq(A, "A_i") == (n, ld)
        mc = len(As)
        ptrs = (ctypes.c_void_p * mc)(*[_ptr(A) for A in As])
        bb = (ctypes.c_double * mc)(*[float(x) for x in b])
        pr = Sdls(_ptr(C), ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)),
                  ctypes.cast(bb, ctypes.POINTER(ctypes.c_double)), n, ld, float(rho), float(beta), float(eps),
                  seed, mc, k, p, q, algorithm, max_iter, int(bool(warm_start)), 0)
        y = (ctypes.c_double * mc)(*[float(v) for v in y0])
        hist = (ctypes.c_double * max_iter)()
        it, gn = _int(), ctypes.c_double()
        _check(_load().psdproj_sdls_dual_gd(self.h, ctypes.byref(pr), y, _ptr(X), X.stride(0) if X is not None else n,
                                            ctypes.byref(it), ctypes.byref(gn), hist,
                                            ctypes.byref(opts) if opts else None), "psdproj_sdls_dual_gd")
        return dict(y=list(y), iters=it.value, gnorm=gn.value, hist=list(hist)[: it.value])

    def tune_batch(self, problems, opts: Opts | None = None, reps: int = 3):
        """psdproj_tune_batch: returns (best lane count, ms per batch)."""
        arr = self._problem_table(problems)
        best, ms = _int(), ctypes.c_double()
        _check(_load().psdproj_tune_batch(self.h, len(problems), ctypes.byref(arr),
                                          ctypes.byref(opts) if opts else None, reps,
                                          ctypes.byref(best), ctypes.byref(ms)), "psdproj_tune_batch")
        return best.value, ms.value

    def set_batch_streams(self, streams: int):
        _check(_load().psdproj_set_batch_streams(self.h, streams), "psdproj_set_batch_streams")

    def set_reserved_sms(self, sms: int):
        _check(_load().psdproj_set_reserved_sms(self.h, sms), "psdproj_set_reserved_sms")

    def alg1_host(self, A, k, p, q, seed, P=None, W=None, opts: Opts | None = None):
        """Host tensors (CPU, pinned recommended); returns r+."""
        n = A.shape[0]
        rk = ctypes.c_int(0)
        _check(_load().psdproj_alg1_host(
            self.h, ctypes.c_void_p(A.data_ptr()), n, A.stride(0), k, p, q, seed,
            _ptr(P), P.stride(0) if P is not None else n, _ptr(W),
            W.stride(1) if W is not None else n, ctypes.byref(rk),
            ctypes.byref(opts) if opts else None), "psdproj_alg1_host")
        return rk.value

    def alg2_host(self, A, k, p, q, seed, alpha_in=0.0, P=None, W=None, opts: Opts | None = None):
        n = A.shape[0]
        rk = ctypes.c_int(0)
        al = ctypes.c_double(0)
        _check(_load().psdproj_alg2_host(
            self.h, ctypes.c_void_p(A.data_ptr()), n, A.stride(0), k, p, q, seed,
            float(alpha_in), ctypes.byref(al), _ptr(P), P.stride(0) if P is not None else n,
            _ptr(W), W.stride(1) if W is not None else n, ctypes.byref(rk),
            ctypes.byref(opts) if opts else None), "psdproj_alg2_host")
        return rk.value, al.value

    # ---- steps of the path -----------------------------------------------
    def gaussian(self, seed, stream_id, X):
        n, m, ld = _tall(X)
        _check(_load().psdproj_gaussian(self.h, seed, stream_id, n, m, _ptr(X), ld), "gaussian")

    def srht(self, seed, X):
        n, m, ld = _tall(X)
        _check(_load().psdproj_srht(self.h, seed, n, m, _ptr(X), ld), "psdproj_srht")

    def sym_pass(self, A, X, Y, shift=None, prec=PREC_FP32):
        n, lda = _sq(A)
        _, m, ldx = _tall(X)
        _, _, ldy = _tall(Y, "Y")
        _check(_load().psdproj_sym_pass(self.h, _ptr(A), n, lda, _ptr(X), ldx, m, _ptr(shift),
                                        _ptr(Y), ldy, prec), "sym_pass")

    def cholqr2(self, Y, Q, qrank=None):
        n, m, ldy = _tall(Y, "Y")
        _, _, ldq = _tall(Q, "Q")
        _check(_load().psdproj_cholqr2(self.h, _ptr(Y), n, ldy, m, _ptr(Q), ldq, _ptr(qrank)),
               "cholqr2")

    def core(self, X, Z, C):
        n, m, ldx = _tall(X)
        _, _, ldz = _tall(Z, "Z")
        _check(_load().psdproj_core(self.h, _ptr(X), ldx, _ptr(Z), ldz, n, m, _ptr(C)), "core")

    def eig(self, C, V, d, method=EIG_AUTO):
        m = C.shape[0]
        _check(_load().psdproj_eig_method(self.h, _ptr(C), m, _ptr(V), _ptr(d), method), "eig")

    def factor(self, Q, V, d, W, rank=None):
        n, m, ldq = _tall(Q, "Q")
        _, _, ldw = _tall(W, "W")
        _check(_load().psdproj_factor(self.h, _ptr(Q), ldq, n, m, _ptr(V), _ptr(d), _ptr(W), ldw,
                                      _ptr(rank)), "factor")

    def syrk(self, W, P, rank=None, out_mode=OUT_FULL, prec=PREC_FP32):
        n, m, ldw = _tall(W, "W")
        _check(_load().psdproj_syrk(self.h, _ptr(W), ldw, n, m, _ptr(rank), _ptr(P), P.stride(0),
                                    out_mode, prec), "syrk")

    def min_eig(self, A, N, seed, alpha, sigma1=None, sigma2=None):
        n, lda = _sq(A)
        _check(_load().psdproj_min_eig(self.h, _ptr(A), n, lda, N, seed, _ptr(alpha),
                                       _ptr(sigma1), _ptr(sigma2)), "min_eig")


class Server:
    """A psdproj_server: requests run by `workers` threads, each with its own
    context and stream, admitted under `admit_bytes` of device memory."""

    def __init__(self, device: int = 0, workers: int = 4, admit_bytes: int = 1 << 34,
                 opts: Opts | None = None):
        h = ctypes.c_void_p()
        _check(_load().psdproj_server_create(ctypes.byref(h), device, workers, admit_bytes,
                                             ctypes.byref(opts) if opts else None), "psdproj_server_create")
        self.h = h
        self._keep = {}

    def submit(self, A, k, p, q, seed, algorithm=1, P=None, W=None, rank=None, alpha_in=0.0,
               alpha_out=None, info=None, footprint_bytes=0) -> int:
        n, lda = _sq(A)
        r = Request(_ptr(A), n, lda, k, p, q, algorithm, seed, float(alpha_in), _ptr(alpha_out), _ptr(info),
                    _ptr(P), P.stride(0) if P is not None else n,
                    _ptr(W), _tall(W, "W")[2] if W is not None else n, _ptr(rank), footprint_bytes)
        t = _u64()
        _check(_load().psdproj_server_submit(self.h, ctypes.byref(r), ctypes.byref(t)), "psdproj_server_submit")
        self._keep[t.value] = (A, P, W, rank, alpha_out, info)   # tensors stay alive until collected
        return t.value

    def wait(self, ticket: int, timeout: float = 60.0):
        """(status, latency_ms) when done, None on timeout."""
        st, lat = _int(), ctypes.c_double()
        rc = _load().psdproj_server_wait(self.h, ticket, timeout, ctypes.byref(st), ctypes.byref(lat))
        if rc == 5:
            return None
        _check(rc, "psdproj_server_wait")
        self._keep.pop(ticket, None)
        return st.value, lat.value

    def drain(self, timeout: float = 600.0):
        _check(_load().psdproj_server_drain(self.h, timeout), "psdproj_server_drain")

    def stats(self) -> dict:
        st = ServerStats()
        _check(_load().psdproj_server_get_stats(self.h, ctypes.byref(st)), "psdproj_server_get_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            _load().psdproj_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_lookup(device_name: str, sm_count: int, median_n: int, count: int):
    """The tuning table's lane count for a batch bucket, or None."""
    v = _int()
    rc = _load().psdproj_tune_lookup(device_name.encode(), sm_count, median_n, count, ctypes.byref(v))
    return v.value if rc == 0 else None


def tune_store(device_name: str, sm_count: int, median_n: int, count: int, streams: int):
    _check(_load().psdproj_tune_store(device_name.encode(), sm_count, median_n, count, streams),
           "psdproj_tune_store")
