"""Python binding of the GoFD C ABI (argument marshalling only).

Device memory and streams come from PyTorch; every step of the method runs in
the CUDA kernels of libgofd.so.  Vectors are torch tensors on the current CUDA
device, in the caller's vertex order (N_v entries) or grid order (n^d entries,
axis 0 fastest).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N


class GofdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{N.STATUS.get(status, status)}: {message}")
        self.status = status
        self.code = N.STATUS.get(status, str(status))


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


_PREC = {"fp64": N.FP64, "fp32": N.FP32, "fp64_df": N.FP64_DF}
_OPS = {"stiffness": N.OP_STIFFNESS, "fraclap": N.OP_FRACLAP}
_MODES = {"fp64": N.SOLVE_FP64, "mixed": N.SOLVE_MIXED}
_RHS = {"grid": N.RHS_GRID, "vertex": N.RHS_VERTEX}


class Problem:
    """One discrete GoFD problem: gofd_build(mesh, alpha, h, box)."""

    def __init__(self, vertices, simplices, alpha: float, h: float, box_lo, box_hi, *, precond: int = 0,
                 ic_level: int = 1, filon_M: int = 0, richardson_levels: int = 0, inner_tol: float = 0.0,
                 check_every: int = 0, wait_budget_cycles: int = 0, ordering: int = 0, chunk_planes: int = 0,
                 fp64_residual: int = 0, ic_solve: int = 0):
        self._lib = N.load()
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        s = np.ascontiguousarray(simplices, dtype=np.int32)
        if v.ndim != 2 or s.ndim != 2 or s.shape[1] != v.shape[1] + 1:
            raise ValueError("vertices must be (N_v, d) and simplices (N_e, d+1)")
        self.d = v.shape[1]
        lo = np.ascontiguousarray(box_lo, dtype=np.float64).reshape(-1)
        hi = np.ascontiguousarray(box_hi, dtype=np.float64).reshape(-1)
        opt = N.Options(precond=precond, ic_level=ic_level, filon_M=filon_M,
                        richardson_levels=richardson_levels, wait_budget_cycles=wait_budget_cycles,
                        inner_tol=inner_tol, check_every=check_every, ordering=ordering,
                        chunk_planes=chunk_planes, fp64_residual=fp64_residual, ic_solve=ic_solve)
        h_ = C.c_void_p()
        st = self._lib.gofd_build(self.d, v.ctypes.data, v.shape[0], s.ctypes.data, s.shape[0], float(alpha),
                                  float(h), lo.ctypes.data, hi.ctypes.data, C.byref(opt), C.byref(h_))
        if st != 0:
            raise GofdError(st, self._lib.gofd_last_error(None).decode())
        self._h = h_
        self.alpha = alpha
        self.h = h
        inf = self.info()
        self.n_v = inf["n_v"]
        self.n_interior = inf["n_interior"]
        self.n = inf["n"][: self.d]
        self.n_grid = inf["n_grid"]
        self.P = inf["P"]

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.gofd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise GofdError(st, self._lib.gofd_last_error(self._h).decode())

    # -- queries ------------------------------------------------------------
    def info(self) -> dict:
        inf = N.Info()
        self._check(self._lib.gofd_get_info(self._h, C.byref(inf)))
        out = {k: getattr(inf, k) for k, _ in N.Info._fields_}
        out["n"] = list(inf.n)
        return out

    def export_transfer(self):
        """(owner[n_grid], ell_idx[d+1, n_loc], ell_w[d+1, n_loc]) as NumPy arrays."""
        inf = self.info()
        nl = inf["n_loc"]
        owner = np.empty(inf["n_grid"], dtype=np.int32)
        idx = np.empty((self.d + 1, nl), dtype=np.int32)
        w = np.empty((self.d + 1, nl), dtype=np.float64)
        self._check(self._lib.gofd_export_transfer(self._h, owner.ctypes.data, idx.ctypes.data, w.ctypes.data))
        return owner, idx, w

    def export_vertex_data(self):
        ii = np.empty(self.n_v, dtype=np.int32)
        cs = np.empty(self.n_v, dtype=np.float64)
        self._check(self._lib.gofd_export_vertex_data(self._h, ii.ctypes.data, cs.ctypes.data))
        return ii, cs

    def export_diagonal(self) -> np.ndarray:
        """The diagonal of S over the interior unknowns (problems built with precond=1)."""
        d = np.empty(self.info()["n_interior"], dtype=np.float64)
        self._check(self._lib.gofd_export_diagonal(self._h, d.ctypes.data))
        return d

    def export_precond(self):
        """(perm, lptr, lcol, lval) of the incomplete Cholesky factor (NumPy)."""
        inf = self.info()
        n, nnz = inf["n_interior"], inf["precond_nnz"]
        perm = np.empty(n, dtype=np.int32)
        lptr = np.empty(n + 1, dtype=np.int32)
        lcol = np.empty(nnz, dtype=np.int32)
        lval = np.empty(nnz, dtype=np.float64)
        self._check(self._lib.gofd_export_precond(self._h, perm.ctypes.data, lptr.ctypes.data, lcol.ctypes.data,
                                                  lval.ctypes.data))
        return perm, lptr, lcol, lval

    def coefficients(self) -> np.ndarray:
        T = np.empty(self.n_grid, dtype=np.float64)
        self._check(self._lib.gofd_get_coefficients(self._h, T.ctypes.data))
        return T.reshape(tuple(reversed(self.n)))

    def symbol(self) -> np.ndarray:
        H = self.P // 2 + 1
        lam = np.empty(H ** self.d, dtype=np.float64)
        self._check(self._lib.gofd_get_symbol(self._h, lam.ctypes.data))
        return lam.reshape((H,) * self.d)

    # -- operators ----------------------------------------------------------
    def apply(self, u, op: str = "stiffness", out=None, stream=None):
        """y = S u (op='stiffness', (GoFD-2)) or h^{-2s} D_h^{-1} S u (op='fraclap')."""
        torch = _torch()
        prec = "fp64" if u.dtype == torch.float64 else "fp32"
        if out is None:
            out = torch.empty_like(u)
        self._check(self._lib.gofd_apply(self._h, _OPS[op], _PREC[prec], _ptr(u), _ptr(out), _stream_ptr(stream)))
        return out

    def apply_interior(self, x, y, stream=None, prec=None):
        """y = S x on interior-compacted vectors.  prec: "fp32" / "fp64" (by
        default from the dtype) or "fp64_df" (float64 vectors, 2D: the FFT
        convolution in double-float arithmetic, as in the mixed solver's
        residual)."""
        torch = _torch()
        if prec is None:
            prec = "fp64" if x.dtype == torch.float64 else "fp32"
        self._check(self._lib.gofd_apply_interior(self._h, _PREC[prec], _ptr(x), _ptr(y), _stream_ptr(stream)))
        return y

    def precond_apply(self, r, z=None, stream=None):
        """z = M^{-1} r with the handle's preconditioner (gofd_precond_apply);
        r: interior-compacted CUDA tensor of N_int + 1 entries (last one 0)."""
        torch = _torch()
        prec = "fp64" if r.dtype == torch.float64 else "fp32"
        if z is None:
            z = torch.empty_like(r)
        self._check(self._lib.gofd_precond_apply(self._h, _PREC[prec], _ptr(r), _ptr(z), _stream_ptr(stream)))
        return z

    def apply_interior_batch(self, X, Y, stream=None):
        """Y[c] = S X[c] for interior-compacted rows (X: nb x ld with ld >= n_int+1
        and X[:, n_int] = 0; Y has the same shape and row stride)."""
        torch = _torch()
        prec = "fp64" if X.dtype == torch.float64 else "fp32"
        if X.dim() != 2 or X.stride(1) != 1 or Y.stride() != X.stride():
            raise TypeError("X and Y must be (nb, ld) with contiguous rows and the same strides")
        self._check(self._lib.gofd_apply_interior_batch(self._h, _PREC[prec], int(X.shape[0]), _ptr(X),
                                                        int(X.stride(0)), _ptr(Y), _stream_ptr(stream)))
        return Y

    def apply_interior_profiled(self, x, y, stream=None):
        """apply_interior with per-stage CUDA-event times: returns [(name, ms), ...]."""
        torch = _torch()
        prec = "fp64" if x.dtype == torch.float64 else "fp32"
        ms = (C.c_float * 32)()
        names = (C.c_char_p * 32)()
        cnt = C.c_int(0)
        self._check(self._lib.gofd_apply_interior_profiled(self._h, _PREC[prec], _ptr(x), _ptr(y),
                                                           _stream_ptr(stream), ms, names, 32, C.byref(cnt)))
        return [(names[i].decode(), float(ms[i])) for i in range(cnt.value)]

    def apply_host(self, u: np.ndarray, op: str = "stiffness", out: np.ndarray | None = None, stream=None):
        """The apply on host buffers: pinned ones are read and written by the
        kernels in place (mapped host memory), pageable ones copied."""
        prec = "fp64" if u.dtype == np.float64 else "fp32"
        u = np.ascontiguousarray(u)
        if out is None:
            out = np.empty_like(u)
        self._check(self._lib.gofd_apply_host(self._h, _OPS[op], _PREC[prec], C.c_void_p(u.ctypes.data),
                                              C.c_void_p(out.ctypes.data), _stream_ptr(stream)))
        return out

    def afd_apply(self, v, out=None, stream=None):
        """w = A_FD v on the grid (Section 2.2)."""
        torch = _torch()
        prec = "fp64" if v.dtype == torch.float64 else "fp32"
        if out is None:
            out = torch.empty_like(v)
        self._check(self._lib.gofd_afd_apply(self._h, _PREC[prec], _ptr(v), _ptr(out), _stream_ptr(stream)))
        return out

    def solve(self, f, rhs: str = "grid", mode: str = "mixed", tol: float = 1e-8, maxit: int = 100000,
              u0=None, stream=None):
        """Solve (GoFD-2); f is a float64 CUDA tensor on the grid or the vertices."""
        torch = _torch()
        if f.dtype != torch.float64:
            raise TypeError("f must be float64")
        u = torch.zeros(self.n_v, dtype=torch.float64, device=f.device) if u0 is None else u0.clone()
        info = N.SolveInfo()
        st = self._lib.gofd_solve(self._h, _MODES[mode], _RHS[rhs], _ptr(f), float(tol), int(maxit),
                                  1 if u0 is None else 0, _ptr(u), C.byref(info), _stream_ptr(stream))
        self._check(st)
        return u, {k: getattr(info, k) for k, _ in N.SolveInfo._fields_}

    def solve_batch(self, F, rhs: str = "grid", mode: str = "mixed", tol: float = 1e-8, maxit: int = 100000,
                    stream=None):
        """Solve S u_c = b_c for the columns of F (nb x n_grid or nb x N_v, float64
        CUDA, rows contiguous) in lock step; returns (U: nb x N_v, infos)."""
        torch = _torch()
        if F.dtype != torch.float64 or F.dim() != 2 or F.stride(1) != 1:
            raise TypeError("F must be a float64 (nb, len) tensor with contiguous rows")
        nb = F.shape[0]
        U = torch.empty((nb, self.n_v), dtype=torch.float64, device=F.device)
        infos = (N.SolveInfo * nb)()
        st = self._lib.gofd_solve_batch(self._h, _MODES[mode], _RHS[rhs], int(nb), _ptr(F), int(F.stride(0)),
                                        float(tol), int(maxit), _ptr(U), C.cast(infos, C.c_void_p),
                                        _stream_ptr(stream))
        self._check(st)
        return U, [{k: getattr(i, k) for k, _ in N.SolveInfo._fields_} for i in infos]

    def autotune(self, nb: int = 1, stream=None) -> float:
        """Pick the fastest launch shapes of the batched product; returns ms per product."""
        ms = C.c_double(0)
        self._check(self._lib.gofd_autotune(self._h, int(nb), _stream_ptr(stream), C.byref(ms)))
        return ms.value

    def set_launch_shapes(self, lines_per_cta: int = 0, cols_per_cta: int = 0, scatter_lanes: int = 0,
                          col_elems: int = 0, row_elems: int = 0, batch_chunk: int = 0) -> None:
        """Set the launch shapes the autotuner chooses from (0 = built-in default)."""
        self._check(self._lib.gofd_set_launch_shapes(self._h, int(lines_per_cta), int(cols_per_cta),
                                                     int(scatter_lanes), int(col_elems), int(row_elems),
                                                     int(batch_chunk)))

    def adjoint(self, f, u, grad_u, mode: str = "mixed", tol: float = 1e-10, maxit: int = 100000, stream=None):
        """(dL/df, dL/dX) for the vertex-data solve u = S^{-1} h^{2s} D_h f given dL/du."""
        torch = _torch()
        gf = torch.empty(self.n_v, dtype=torch.float64, device=f.device)
        gx = torch.empty((self.n_v, self.d), dtype=torch.float64, device=f.device)
        info = N.SolveInfo()
        g = grad_u.to(torch.float64).contiguous()
        self._check(self._lib.gofd_adjoint(self._h, _MODES[mode], _ptr(f.contiguous()), _ptr(u.contiguous()),
                                           _ptr(g), float(tol), int(maxit), _ptr(gf), _ptr(gx), C.byref(info),
                                           _stream_ptr(stream)))
        return gf, gx, {k: getattr(info, k) for k, _ in N.SolveInfo._fields_}


class Group:
    """Several 2D problems on one overlay grid, nb right-hand sides each,
    solved together in lock step (gofd_group_*): one block PCG over all
    columns, one CUDA graph launch per inner solve, every product kernel
    covering all problems' columns.  The problems must outlive the group."""

    def __init__(self, problems, nb: int):
        self._lib = N.load()
        self.problems = list(problems)
        self.nb = int(nb)
        arr = (C.c_void_p * len(self.problems))(*[q._h.value for q in self.problems])
        h = C.c_void_p()
        st = self._lib.gofd_group_create(len(self.problems), C.cast(arr, C.c_void_p), self.nb, C.byref(h))
        if st != 0:
            raise GofdError(st, self._lib.gofd_last_error(None).decode())
        self._g = h

    def _check(self, st: int):
        if st != 0:
            raise GofdError(st, self._lib.gofd_last_error(None).decode())

    def autotune(self, stream=None) -> float:
        """Tune the launch shapes of the group's product; returns ms per product."""
        ms = C.c_double(0)
        self._check(self._lib.gofd_group_autotune(self._g, _stream_ptr(stream), C.byref(ms)))
        return ms.value

    def solve(self, batches, rhs: str = "grid", mode: str = "mixed", tol: float = 1e-8, maxit: int = 100000,
              stream=None):
        """batches[i]: (nb, len) float64 CUDA tensor of problem i (rows contiguous).
        Returns [(U_i: nb x N_v(i), infos_i)] in the problems' order."""
        torch = _torch()
        np_ = len(self.problems)
        if len(batches) != np_:
            raise ValueError("one batch per problem")
        Us = []
        for q, F in zip(self.problems, batches):
            if F.dtype != torch.float64 or F.dim() != 2 or F.shape[0] != self.nb or F.stride(1) != 1:
                raise TypeError("each batch must be a float64 (nb, len) tensor with contiguous rows")
            Us.append(torch.empty((self.nb, q.n_v), dtype=torch.float64, device=F.device))
        fp = (C.c_void_p * np_)(*[F.data_ptr() for F in batches])
        up = (C.c_void_p * np_)(*[U.data_ptr() for U in Us])
        ld = (C.c_int64 * np_)(*[int(F.stride(0)) for F in batches])
        infos = (N.SolveInfo * (np_ * self.nb))()
        self._check(self._lib.gofd_group_solve(self._g, _MODES[mode], _RHS[rhs], C.cast(fp, C.c_void_p),
                                               C.cast(ld, C.c_void_p), float(tol), int(maxit),
                                               C.cast(up, C.c_void_p), C.cast(infos, C.c_void_p),
                                               _stream_ptr(stream)))
        rows = [{k: getattr(i, k) for k, _ in N.SolveInfo._fields_} for i in infos]
        return [(Us[i], rows[i * self.nb:(i + 1) * self.nb]) for i in range(np_)]

    def close(self):
        if getattr(self, "_g", None):
            self._lib.gofd_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_key(problem):
    """Problems with equal keys share an overlay grid (and can form a Group)."""
    inf = problem.info()
    return (inf["d"], tuple(inf["n"]), inf["P"], float(problem.h))


def group_key(problem):
    """The partition solve_many uses: one overlay grid and one alpha.  Columns
    of one alpha need similar iteration counts (the condition number grows
    with alpha), so a lock-step group wastes little on columns that finish
    early, and its members share one symbol."""
    return grid_key(problem) + (float(problem.alpha),)


def solve_many(problems, batches, rhs: str = "grid", mode: str = "mixed", tol: float = 1e-8,
               maxit: int = 100000, groups=None):
    """Independent problems solved together.  2D problems are grouped by grid
    and alpha (group_key): each group is solved as one Group (all its columns
    in one block PCG); groups, and problems of other dimensions (solve_batch),
    run concurrently, one host thread and stream each (the C calls release
    the interpreter lock).  groups: optional dict group_key -> Group built
    earlier for these problems (reused; keeps its tuned launch shapes).
    Returns the list of (U, infos) in the problems' order."""
    import threading
    torch = _torch()
    dev = torch.cuda.current_device()
    units = {}
    for i, q in enumerate(problems):
        key = group_key(q) if q.d == 2 else ("single", i)
        units.setdefault(key, []).append(i)
    keys = list(units)
    nb = {i: batches[i].shape[0] for i in range(len(problems))}
    # groups this call builds: made here, before any worker starts, and closed
    # after every worker has returned -- creating or destroying a handle
    # allocates or frees device memory, and a free synchronises the device,
    # which would break another worker's CUDA graph capture
    own = {}
    for key in keys:
        idx = units[key]
        if key[0] != "single" and len(set(nb[i] for i in idx)) == 1 and not (groups and key in groups):
            own[key] = Group([problems[i] for i in idx], nb[idx[0]])
    streams = [torch.cuda.Stream() for _ in keys]
    for s in streams:
        s.wait_stream(torch.cuda.current_stream())
    out = [None] * len(problems)
    errs = [None] * len(keys)

    def work(u):
        try:
            torch.cuda.set_device(dev)
            idx = units[keys[u]]
            with torch.cuda.stream(streams[u]):
                g = own.get(keys[u]) or (groups.get(keys[u]) if groups else None)
                if g is None:
                    for i in idx:
                        out[i] = problems[i].solve_batch(batches[i], rhs=rhs, mode=mode, tol=tol, maxit=maxit,
                                                         stream=streams[u])
                    return
                res = g.solve([batches[i] for i in idx], rhs=rhs, mode=mode, tol=tol, maxit=maxit,
                              stream=streams[u])
                for i, r in zip(idx, res):
                    out[i] = r
        except Exception as e:  # re-raised on the caller's thread
            errs[u] = e

    threads = [threading.Thread(target=work, args=(u,)) for u in range(len(keys))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for s in streams:
        torch.cuda.current_stream().wait_stream(s)
    for g in own.values():
        g.close()
    for e in errs:
        if e is not None:
            raise e
    return out


def fma_rates(stream=None):
    """Measured FP64 and FP32 FMA throughput of the current device (GFLOP/s)."""
    lib = N.load()
    f64, f32 = C.c_double(0), C.c_double(0)
    st = lib.gofd_fma_rates(_stream_ptr(stream), C.byref(f64), C.byref(f32))
    if st != 0:
        raise GofdError(st, "gofd_fma_rates failed")
    return f64.value, f32.value


def afd_apply_noalloc(d: int, n: int, lam_scaled, v, out=None, stream=None):
    """w = A_FD v (FP32) through the entry point that allocates nothing.

    For callers that cannot allocate device memory when they need the product
    (under a framework that owns all device memory, in real-time loops that
    must not risk an allocation failure or its latency): the library keeps its
    scratch in a fixed device array.
    lam_scaled is the float32 symbol lambda_k / P^d on [0, P/2]^d; v and out
    are float32 grid vectors of n^d entries.  Calls that overlap on the GPU
    race on the shared scratch.
    """
    lib = N.load()
    torch = _torch()
    if out is None:
        out = torch.empty_like(v)
    st = lib.gofd_afd_apply_noalloc(int(d), int(n), _ptr(lam_scaled), _ptr(v), _ptr(out), _stream_ptr(stream))
    if st != 0:
        raise GofdError(st, lib.gofd_last_error(None).decode())
    return out


class _SolveFunction:
    """torch.autograd.Function for u = S(X)^{-1} h^{2s} D_h(X) f (vertex data)."""

    _fn = None

    @classmethod
    def get(cls):
        if cls._fn is None:
            torch = _torch()

            class Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, f, X, simplices, alpha, h, box_lo, box_hi, tol, mode, opts):
                    prob = Problem(X.detach().cpu().numpy(), simplices, alpha, h, box_lo, box_hi, **opts)
                    fd = f.detach().to(torch.float64).contiguous()
                    u, _ = prob.solve(fd, rhs="vertex", mode=mode, tol=tol)
                    ctx.prob, ctx.tol, ctx.mode = prob, tol, mode
                    ctx.save_for_backward(fd, u)
                    return u

                @staticmethod
                def backward(ctx, grad_u):
                    fd, u = ctx.saved_tensors
                    gf, gx, _ = ctx.prob.adjoint(fd, u, grad_u, mode=ctx.mode, tol=ctx.tol)
                    ctx.prob.close()
                    return gf, gx, None, None, None, None, None, None, None, None

            cls._fn = Fn
        return cls._fn


def solve(f, X, simplices, alpha, h, box_lo, box_hi, tol: float = 1e-10, mode: str = "mixed", **opts):
    """Differentiable solve of (GoFD-3): returns u (N_v) for vertex data f (N_v)
    and vertex coordinates X (N_v x d), both CUDA tensors; gradients flow to f
    and X through the adjoint (the owner map of the grid nodes is held fixed)."""
    return _SolveFunction.get().apply(f, X, simplices, alpha, h, box_lo, box_hi, tol, mode, opts)
