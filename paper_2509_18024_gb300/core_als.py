"""Python front end of the CUDA Core-ALS library.

PyTorch supplies device memory and the current CUDA stream; every step of the
half-sweep (CES selection, Gram assembly, solve) runs in libcore_als.so. This
module only moves arguments across the C ABI (see binding.py).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B

GRAM_MODES = {"asym": B.ALS_GRAM_ASYM, "sym": B.ALS_GRAM_SYM, "full": B.ALS_GRAM_FULL}
SKETCHES = {"slice": B.ALS_SKETCH_SLICE, "factor": B.ALS_SKETCH_FACTOR}
REG_MODES = {"weighted": B.ALS_REG_WEIGHTED, "plain": B.ALS_REG_PLAIN}


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required: libcore_als.so has no CPU path")


@dataclass
class DeviceCSR:
    """One side of the rating matrix on the device (CSR of R or of R^T)."""
    n_rows: int
    n_cols: int
    indptr: torch.Tensor   # int64
    indices: torch.Tensor  # int32
    values: torch.Tensor   # float32

    @property
    def nnz(self) -> int:
        return int(self.indices.shape[0])

    @classmethod
    def from_host(cls, csr, device="cuda") -> "DeviceCSR":
        return cls(int(csr.n_rows), int(csr.n_cols),
                   torch.as_tensor(np.ascontiguousarray(csr.indptr, np.int64)).to(device),
                   torch.as_tensor(np.ascontiguousarray(csr.indices, np.int32)).to(device),
                   torch.as_tensor(np.ascontiguousarray(csr.values, np.float32)).to(device))

    def c_struct(self) -> B.als_csr:
        return B.als_csr(self.n_rows, self.n_cols, self.nnz, self.indptr.data_ptr(),
                         self.indices.data_ptr() if self.nnz else None,
                         self.values.data_ptr() if self.nnz else None)


class CoreALS:
    """A handle of the CUDA library with fixed options."""

    def __init__(self, n_f: int, lam: float, budget: float, gram_mode: str = "asym",
                 reg_mode: str = "weighted", min_keep: int = 0, ratio_max: float = 1e6,
                 precision: int = B.ALS_FP32, fp64_fallback: bool = True, refine_steps: int = B.ALS_REFINE_AUTO,
                 fixed_keep: int = 0, sketch: str = "slice"):
        _require_cuda()
        self.lib = B.load()
        opt = B.als_options()
        self.lib.als_default_options(C.byref(opt))
        opt.n_f = int(n_f)
        opt.lambda_ = float(lam)
        opt.budget = float(budget)
        opt.min_keep = int(min_keep)
        opt.reg_mode = REG_MODES[reg_mode]
        opt.gram_mode = GRAM_MODES[gram_mode]
        opt.precision = int(precision)
        opt.pivot_ratio_max = float(ratio_max)
        opt.fp64_fallback = 1 if fp64_fallback else 0
        opt.refine_steps = int(refine_steps)
        opt.fixed_keep = int(fixed_keep)
        opt.sketch = SKETCHES[sketch]
        self.opt = opt
        self.n_f = int(n_f)
        h = C.c_void_p()
        B.check(self.lib.als_create(C.byref(h), C.byref(opt), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        self.h = h

    # -- plumbing -----------------------------------------------------------
    def _bind_stream(self):
        B.check(self.lib.als_set_stream(self.h, C.c_void_p(torch.cuda.current_stream().cuda_stream)), self.h)

    def _call(self, fn, *args):
        self._bind_stream()
        B.check(fn(self.h, *args), self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.als_destroy(self.h)
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

    @property
    def launch_count(self) -> int:
        return int(self.lib.als_launch_count(self.h))

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.als_workspace_bytes(self.h))

    # -- the calls ----------------------------------------------------------
    def prepare(self, R: DeviceCSR):
        self._call(self.lib.als_prepare, C.byref(R.c_struct()))

    def half_sweep(self, R: DeviceCSR, Y: torch.Tensor, X: torch.Tensor | None = None,
                   flags: torch.Tensor | None = None):
        """One half-sweep of Algorithm 2: X (R.n_rows x n_f) from Y (R.n_cols x n_f)."""
        if X is None:
            X = torch.empty((R.n_rows, self.n_f), dtype=torch.float32, device=Y.device)
        self._call(self.lib.als_half_sweep, C.byref(R.c_struct()), B.ptr(Y), B.ptr(X), B.ptr(flags))
        return X

    def select(self, R: DeviceCSR, Y: torch.Tensor) -> torch.Tensor:
        """CES masks as int32[nnz, ceil(n_f/32)] (bit patterns of uint32 words)."""
        words = (self.n_f + 31) // 32
        masks = torch.zeros((R.nnz, words), dtype=torch.int32, device=Y.device)
        self._call(self.lib.als_select, C.byref(R.c_struct()), B.ptr(Y), B.ptr(masks))
        return masks

    def assemble(self, R: DeviceCSR, Y: torch.Tensor):
        G = torch.zeros((R.n_rows, self.n_f, self.n_f), dtype=torch.float32, device=Y.device)
        b = torch.zeros((R.n_rows, self.n_f), dtype=torch.float32, device=Y.device)
        self._call(self.lib.als_assemble, C.byref(R.c_struct()), B.ptr(Y), B.ptr(G), B.ptr(b))
        return G, b

    def solve(self, G: torch.Tensor, b: torch.Tensor):
        n = int(b.shape[0])
        X = torch.empty((n, self.n_f), dtype=torch.float32, device=b.device)
        flags = torch.empty(n, dtype=torch.int32, device=b.device)
        self._call(self.lib.als_solve, n, B.ptr(G.contiguous()), B.ptr(b.contiguous()), B.ptr(X), B.ptr(flags))
        return X, flags

    def sse(self, iu: torch.Tensor, im: torch.Tensor, r: torch.Tensor, U: torch.Tensor, M: torch.Tensor) -> float:
        out = C.c_double()
        self._call(self.lib.als_eval_sse, int(r.shape[0]), B.ptr(iu), B.ptr(im), B.ptr(r), B.ptr(U), B.ptr(M),
                   C.byref(out))
        return out.value

    def rmse(self, iu, im, r, U, M) -> float:
        n = int(r.shape[0])
        return float(np.sqrt(self.sse(iu, im, r, U, M) / n)) if n else 0.0

    def sse_async(self, iu, im, r, U, M, out: torch.Tensor):
        """Enqueue the SSE into out (a float64 device tensor of one element)."""
        self._call(self.lib.als_eval_sse_async, int(r.shape[0]), B.ptr(iu), B.ptr(im), B.ptr(r), B.ptr(U),
                   B.ptr(M), B.ptr(out))

    def objective(self, Ru: DeviceCSR, Ri: DeviceCSR, U: torch.Tensor, M: torch.Tensor) -> float:
        """Eq. (object function) at (U, M) with the handle's lambda and regulariser."""
        out = C.c_double()
        self._call(self.lib.als_objective, C.byref(Ru.c_struct()), C.byref(Ri.c_struct()), B.ptr(U), B.ptr(M),
                   C.byref(out))
        return out.value

    def remse(self, iu, im, r, U, M) -> float:
        """Sec. 5.1 relative error over the listed entries (ReMSE / P-ReMSE)."""
        out = C.c_double()
        self._call(self.lib.als_eval_remse, int(r.shape[0]), B.ptr(iu), B.ptr(im), B.ptr(r), B.ptr(U), B.ptr(M),
                   C.byref(out))
        return out.value

    def ranking(self, R_train: DeviceCSR, rel: DeviceCSR, U, M, k_hit: int = 5, k_ndcg: int = 10,
                want_lists: bool = False):
        """(Hit@k_hit, NDCG@k_ndcg, users evaluated[, lists]) of Sec. 5.1."""
        K = max(k_hit, k_ndcg)
        lists = torch.empty((R_train.n_rows, K), dtype=torch.int32, device=U.device) if want_lists else None
        hit, ndcg, n = C.c_double(), C.c_double(), C.c_int64()
        self._call(self.lib.als_eval_ranking, C.byref(R_train.c_struct()), C.byref(rel.c_struct()), B.ptr(U),
                   B.ptr(M), int(k_hit), int(k_ndcg), B.ptr(lists), C.byref(hit), C.byref(ndcg), C.byref(n))
        out = (hit.value, ndcg.value, n.value)
        return out + (lists,) if want_lists else out

    def profile(self, enable: bool = True):
        """als_profile: time every launch with CUDA events (half-sweeps then
        run on the handle's stream alone, without side streams)."""
        self._call(self.lib.als_profile, 1 if enable else 0)

    def kernel_time(self, family: str | None = None):
        """(summed CUDA-event ms, launches) of one kernel family since profile()."""
        ms = C.c_double()
        n = C.c_int64()
        self._call(self.lib.als_kernel_time, family.encode() if family else None, C.byref(ms), C.byref(n))
        return ms.value, n.value

    def autotune(self, Ru: DeviceCSR, Ri: DeviceCSR, U: torch.Tensor, M: torch.Tensor, trials: int = 3) -> dict:
        """Time the candidate schedules on this problem and keep the fastest."""
        t = B.als_tuning()
        self._call(self.lib.als_autotune, C.byref(Ru.c_struct()), C.byref(Ri.c_struct()), B.ptr(U), B.ptr(M),
                   int(trials), C.byref(t))
        return {k: getattr(t, k) for k, _ in B.als_tuning._fields_}

    def set_tuning(self, split_at_middle=0, warp_rows=1, tc_gram=0):
        t = B.als_tuning(int(split_at_middle), int(warp_rows), int(tc_gram), 0.0)
        self._call(self.lib.als_set_tuning, C.byref(t))

    def report(self) -> dict:
        rep = B.als_report()
        self._call(self.lib.als_get_report, C.byref(rep))
        return {k: getattr(rep, k) for k, _ in B.als_report._fields_}

    def sweep(self, Ru: DeviceCSR, Ri: DeviceCSR, U: torch.Tensor, M: torch.Tensor):
        self._call(self.lib.als_sweep, C.byref(Ru.c_struct()), C.byref(Ri.c_struct()), B.ptr(U), B.ptr(M))

    def fit(self, Ru: DeviceCSR, Ri: DeviceCSR, M0: torch.Tensor, sweeps: int, test=None):
        """Algorithm 2 from M^(0) = M0 (copied). test = (iu, im, r) device tensors or None."""
        M = M0.clone()
        U = torch.empty((Ru.n_rows, self.n_f), dtype=torch.float32, device=M.device)
        rep = B.als_report()
        if test is not None:
            iu, im, r = test
            n_test, tp = int(r.shape[0]), (B.ptr(iu), B.ptr(im), B.ptr(r))
        else:
            n_test, tp = 0, (None, None, None)
        self._call(self.lib.als_fit, C.byref(Ru.c_struct()), C.byref(Ri.c_struct()), int(sweeps), B.ptr(U),
                   B.ptr(M), n_test, *tp, C.byref(rep))
        return U, M, {k: getattr(rep, k) for k, _ in B.als_report._fields_}

    def fit_host(self, rows, cols, M0: np.ndarray, sweeps: int, test=None):
        """als_fit_host: every input and output in host memory (numpy arrays)."""
        U = np.zeros((rows.n_rows, self.n_f), np.float32)
        M = np.ascontiguousarray(M0, np.float32).copy()
        hold = []

        def hp(a, dt):
            a = np.ascontiguousarray(a, dt)
            hold.append(a)
            return a.ctypes.data_as(C.c_void_p)

        rep = B.als_report()
        if test is not None:
            tu, tm, tr = test
            n_test, tp = len(tr), (hp(tu, np.int32), hp(tm, np.int32), hp(tr, np.float32))
        else:
            n_test, tp = 0, (None, None, None)
        self._call(self.lib.als_fit_host, rows.n_rows, cols.n_rows, int(rows.indices.shape[0]),
                   hp(rows.indptr, np.int64), hp(rows.indices, np.int32), hp(rows.values, np.float32),
                   hp(cols.indptr, np.int64), hp(cols.indices, np.int32), hp(cols.values, np.float32),
                   int(sweeps), U.ctypes.data_as(C.c_void_p), M.ctypes.data_as(C.c_void_p), n_test, *tp,
                   C.byref(rep))
        return U, M, {k: getattr(rep, k) for k, _ in B.als_report._fields_}


class CoreBatch:
    """Independent completion problems fitted together (als_batch_*).

    problems: list of (DeviceCSR users, DeviceCSR items, n_f, U, M) with U, M
    device tensors (M holds M^(0) and receives the result). Options other
    than n_f are shared. The stream is a new CUDA stream unless given.
    """

    def __init__(self, problems, lam: float, budget: float, gram_mode: str = "asym", reg_mode: str = "weighted",
                 precision: int = B.ALS_FP32, fp64_fallback: bool = True, refine_steps: int = B.ALS_REFINE_AUTO,
                 stream=None, fixed_keep: int = 0, sketch: str = "slice"):
        _require_cuda()
        self.lib = B.load()
        opt = B.als_options()
        self.lib.als_default_options(C.byref(opt))
        opt.lambda_ = float(lam)
        opt.budget = float(budget)
        opt.reg_mode = REG_MODES[reg_mode]
        opt.gram_mode = GRAM_MODES[gram_mode]
        opt.precision = int(precision)
        opt.fp64_fallback = 1 if fp64_fallback else 0
        opt.refine_steps = int(refine_steps)
        opt.fixed_keep = int(fixed_keep)
        opt.sketch = SKETCHES[sketch]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.problems = problems  # keep the tensors alive
        arr = (B.als_problem * len(problems))()
        for q, (Ru, Ri, n_f, U, M) in enumerate(problems):
            arr[q] = B.als_problem(Ru.c_struct(), Ri.c_struct(), int(n_f), U.data_ptr(), M.data_ptr())
        b = C.c_void_p()
        torch.cuda.current_stream().synchronize()
        B.check(self.lib.als_batch_create(C.byref(b), C.byref(opt), len(problems), arr,
                                          C.c_void_p(self.stream.cuda_stream)))
        self.b = b

    @property
    def launches_per_sweep(self) -> int:
        return int(self.lib.als_batch_launches_per_sweep(self.b))

    def select(self, q: int, side: int, Y: torch.Tensor) -> torch.Tensor:
        """CES masks of problem q's side (0 users, 1 items) from the batched
        structure, with that problem's design factor Y."""
        Ru, Ri, n_f = self.problems[q][:3]
        masks = torch.zeros(((Ru if side == 0 else Ri).nnz, (n_f + 31) // 32), dtype=torch.int32, device=Y.device)
        B.check(self.lib.als_batch_select(self.b, int(q), int(side), B.ptr(Y.contiguous()), B.ptr(masks)))
        return masks

    def fit(self, sweeps: int):
        B.check(self.lib.als_batch_fit(self.b, int(sweeps)))
        return self

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "b", None):
            self.lib.als_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe(kind: str):
    """(rate, ms) of one roofline probe (als_probe): TFLOP/s for ffma, dfma,
    tc_bf16, tc_tf32; GB/s for l2_gather and hbm_copy."""
    _require_cuda()
    lib = B.load()
    v, ms = C.c_double(), C.c_double()
    B.check(lib.als_probe(B.PROBES[kind], C.byref(v), C.byref(ms),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return v.value, ms.value


def features(R: DeviceCSR, Y: torch.Tensor, n_f: int) -> torch.Tensor:
    """Per-row warm-start features of one side (n_rows x (n_f + 2))."""
    lib = B.load()
    out = torch.empty((R.n_rows, n_f + 2), dtype=torch.float32, device=Y.device)
    B.check(lib.als_features(C.byref(R.c_struct()), B.ptr(Y), int(n_f), B.ptr(out),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


class MLP:
    """The warm-start network (als_mlp_*): in -> hidden -> hidden -> out, GELU."""

    def __init__(self, in_dim: int, hidden: int, out_dim: int, seed: int = 0):
        _require_cuda()
        self.lib = B.load()
        self.dims = (in_dim, hidden, out_dim)
        m = C.c_void_p()
        B.check(self.lib.als_mlp_create(C.byref(m), int(in_dim), int(hidden), int(out_dim), int(seed),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        self.m = m
        self.n_params = int(self.lib.als_mlp_num_params(m))

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        B.check(self.lib.als_mlp_get_params(self.m, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        B.check(self.lib.als_mlp_set_params(self.m, p.ctypes.data_as(C.c_void_p)))

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        X = X.contiguous()
        Y = torch.empty((X.shape[0], self.dims[2]), dtype=torch.float32, device=X.device)
        B.check(self.lib.als_mlp_forward(self.m, int(X.shape[0]), B.ptr(X), B.ptr(Y)))
        return Y

    def grad(self, X: torch.Tensor, T: torch.Tensor):
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_double()
        B.check(self.lib.als_mlp_grad(self.m, int(X.shape[0]), B.ptr(X.contiguous()), B.ptr(T.contiguous()),
                                      g.ctypes.data_as(C.c_void_p), C.byref(loss)))
        return loss.value, g

    def train_step(self, X: torch.Tensor, T: torch.Tensor, lr: float, want_loss: bool = False):
        loss = C.c_double()
        B.check(self.lib.als_mlp_train_step(self.m, int(X.shape[0]), B.ptr(X), B.ptr(T), float(lr),
                                            C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "m", None):
            self.lib.als_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
