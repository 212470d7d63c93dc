"""GB300 Recursive Schur Decomposition preconditioner: Python binding of include/rsd.h.

Thin marshalling over the C ABI (librsd.so).  PyTorch provides device memory and the
stream; every step of setup, apply and solve runs in the library's CUDA kernels.

    prob = grid_problem(n, depth, kappa, f)           # K, b, ownership, tree on the GPU
    h = RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"])
    u, stats = h.solve(prob["b"], tol=1e-8)
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (RSD_KRYLOV_AUTO, RSD_KRYLOV_FGMRES, RSD_KRYLOV_PCG, RSD_MEM_DEVICE, RSD_MEM_HOST,
                   RSD_MODE_EXACT, RSD_MODE_PAPER, RSD_PREC_BF16, RSD_PREC_FP16, RSD_PREC_FP32, RSD_PREC_FP64,
                   RSD_PREC_TF32, RSDError, check)

__all__ = ["RSD", "grid_problem", "grid_problem_elastic", "grid_sizes", "grid_exp", "coef_grad", "diffusion_solve",
           "DiffusionSolve", "launch_count", "peak_gemm", "autotune", "tune_entries", "RSDError", "RSD_PREC_FP64", "RSD_PREC_FP32",
           "RSD_PREC_TF32", "RSD_PREC_FP16", "RSD_PREC_BF16", "RSD_MODE_EXACT", "RSD_MODE_PAPER", "RSD_KRYLOV_AUTO", "RSD_KRYLOV_PCG",
           "RSD_KRYLOV_FGMRES"]


def peak_gemm(prec: int, n: int, reps: int = 5, seconds: float = 4.0) -> tuple[float, float]:
    """(best, sustained) TFLOP/s of the library's own GEMM kernel for `prec` on an
    n x n x n product (rsd_peak_gemm), on the current stream."""
    best, sus = C.c_double(), C.c_double()
    check(_lib.load().rsd_peak_gemm(prec, n, reps, seconds, _stream(), C.byref(best), C.byref(sus)),
          "rsd_peak_gemm")
    return best.value, sus.value


def autotune(path: str) -> float:
    """Time the tensor-core GEMM configurations per size bucket and write the fastest to
    `path` (rsd_autotune); returns the seconds taken.  Pass the path as tune_cache to
    RSD.setup to use it."""
    secs = C.c_double()
    check(_lib.load().rsd_autotune(path.encode(), C.byref(secs), _stream()), "rsd_autotune")
    return secs.value


def tune_entries(path: str) -> int:
    """Number of buckets in a table written by autotune (rsd_tune_load; host only)."""
    n = C.c_int32()
    check(_lib.load().rsd_tune_load(path.encode(), C.byref(n)), "rsd_tune_load")
    return n.value


def launch_count() -> int:
    """Kernels librsd has launched in this process."""
    return int(_lib.load().rsd_launch_count())


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def grid_sizes(n: int) -> tuple[int, int]:
    lib = _lib.load()
    nd, nz = C.c_int64(), C.c_int64()
    check(lib.rsd_grid_sizes(n, C.byref(nd), C.byref(nz)), "rsd_grid_sizes")
    return nd.value, nz.value


def grid_problem(n: int, depth: int, kappa, f, device: str = "cuda") -> dict:
    """Assemble K (CSR, FP64), b = h^3 f, the octree ownership and tree on the GPU.
    kappa: (n-1)^3 per-element coefficients; f: (n-2)^3 nodal loads."""
    lib = _lib.load()
    nd, _ = grid_sizes(n)
    kap = torch.as_tensor(np.ascontiguousarray(kappa), dtype=torch.float64).to(device)
    fn = torch.as_tensor(np.ascontiguousarray(f), dtype=torch.float64).to(device)
    prob = _grid_system(n, depth, kap)
    b = torch.empty(nd, dtype=torch.float64, device=device)
    check(lib.rsd_grid_load(n, _ptr(fn), _ptr(b), _stream()), "rsd_grid_load")
    prob["b"] = b
    return prob


def grid_problem_elastic(n: int, depth: int, E_leaf, nu: float, f, device: str = "cuda") -> dict:
    """3-D linear elasticity on the n^3 grid (three DOFs per node): K with Young's modulus
    E_leaf[l] on octree leaf l (8^depth values) and Poisson's ratio nu, b = h^3 f (f per
    DOF, 3 (n-2)^3 values), the ownership (each DOF owned by its node's owner) and tree."""
    lib = _lib.load()
    nd, nz = C.c_int64(), C.c_int64()
    check(lib.rsd_grid_elastic_sizes(n, C.byref(nd), C.byref(nz)), "rsd_grid_elastic_sizes")
    nd, nz = nd.value, nz.value
    E = torch.as_tensor(np.ascontiguousarray(E_leaf), dtype=torch.float64).to(device)
    fn = torch.as_tensor(np.ascontiguousarray(f), dtype=torch.float64).to(device)
    rowptr = torch.empty(nd + 1, dtype=torch.int64, device=device)
    col = torch.empty(nz, dtype=torch.int32, device=device)
    val = torch.empty(nz, dtype=torch.float64, device=device)
    dof_node = torch.empty(nd, dtype=torch.int32, device=device)
    scratch = torch.empty(nd // 3, dtype=torch.int32, device=device)
    n_nodes = (8 ** (depth + 1) - 1) // 7
    parent = np.empty(n_nodes, dtype=np.int32)
    b = torch.empty(nd, dtype=torch.float64, device=device)
    st = _stream()
    check(lib.rsd_grid_elastic_assemble(n, depth, _ptr(E), nu, _ptr(rowptr), _ptr(col), _ptr(val), st),
          "rsd_grid_elastic_assemble")
    check(lib.rsd_grid_elastic_partition(n, depth, _ptr(dof_node), parent.ctypes.data, _ptr(scratch), st),
          "rsd_grid_elastic_partition")
    check(lib.rsd_grid_elastic_load(n, _ptr(fn), _ptr(b), st), "rsd_grid_elastic_load")
    return dict(n=n, depth=depth, n_dof=nd, nnz=nz, rowptr=rowptr, col=col, val=val,
                dof_node=dof_node, parent=parent, b=b)


def _grid_system(n: int, depth: int, kappa: torch.Tensor) -> dict:
    """K(kappa) in CSR and the octree ownership, assembled on kappa's device."""
    lib = _lib.load()
    nd, nz = grid_sizes(n)
    device = kappa.device
    rowptr = torch.empty(nd + 1, dtype=torch.int64, device=device)
    col = torch.empty(nz, dtype=torch.int32, device=device)
    val = torch.empty(nz, dtype=torch.float64, device=device)
    dof_node = torch.empty(nd, dtype=torch.int32, device=device)
    n_nodes = (8 ** (depth + 1) - 1) // 7
    parent = np.empty(n_nodes, dtype=np.int32)
    st = _stream()
    check(lib.rsd_grid_assemble(n, _ptr(kappa), _ptr(rowptr), _ptr(col), _ptr(val), st), "rsd_grid_assemble")
    check(lib.rsd_grid_partition(n, depth, _ptr(dof_node), parent.ctypes.data, st), "rsd_grid_partition")
    return dict(n=n, depth=depth, n_dof=nd, nnz=nz, rowptr=rowptr, col=col, val=val,
                dof_node=dof_node, parent=parent)


def grid_exp(n: int, m: torch.Tensor) -> torch.Tensor:
    """kappa = exp(m) per element, on the device (rsd_grid_exp)."""
    m = m.to(torch.float64).contiguous()
    kappa = torch.empty_like(m)
    check(_lib.load().rsd_grid_exp(n, _ptr(m), _ptr(kappa), _stream()), "rsd_grid_exp")
    return kappa


def coef_grad(n: int, u: torch.Tensor, lam: torch.Tensor, kappa: torch.Tensor | None = None):
    """Per-element dL/dkappa = -lam_e^T K_e u_e and, given kappa, dL/dm = kappa * dL/dkappa
    (rsd_grid_coef_grad).  Returns (dkappa, dm or None)."""
    ne3 = (n - 1) ** 3
    dk = torch.empty(ne3, dtype=torch.float64, device=u.device)
    dm = torch.empty_like(dk) if kappa is not None else None
    check(_lib.load().rsd_grid_coef_grad(n, _ptr(u), _ptr(lam), _ptr(kappa) if kappa is not None else None,
                                         _ptr(dk), _ptr(dm) if dm is not None else None, _stream()),
          "rsd_grid_coef_grad")
    return dk, dm


class RSD:
    """A built hierarchy (rsd_handle).  Use RSD.setup(...)."""

    def __init__(self, handle: int, n: int):
        self._h = C.c_void_p(handle)
        self.n = n

    @classmethod
    def setup(cls, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
              dof_node: torch.Tensor, parent, prec_leaf: int = RSD_PREC_TF32,
              prec_mid: int = RSD_PREC_TF32, prec_root: int = RSD_PREC_FP64,
              maxit: int = 200, profile: bool = False, mode: int = RSD_MODE_EXACT,
              wait_cycles: int = 0, gamma: int = 0, krylov: int = 0, restart: int = 0,
              tune_cache: str | None = None, nonsymmetric: bool = False) -> "RSD":
        lib = _lib.load()
        dev = rowptr.is_cuda
        if not (col.is_cuda == dev and val.is_cuda == dev and dof_node.is_cuda == dev):
            raise ValueError("rowptr, col, val and dof_node must all be on the device or all on the host")
        rowptr = rowptr.to(torch.int64).contiguous()
        col = col.to(torch.int32).contiguous()
        val = val.to(torch.float64).contiguous()
        dof_node = dof_node.to(torch.int32).contiguous()
        par = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
        n = rowptr.numel() - 1
        csr = _lib.rsd_csr(n, col.numel(), _ptr(rowptr), _ptr(col), _ptr(val),
                           RSD_MEM_DEVICE if dev else RSD_MEM_HOST)
        tree = _lib.rsd_tree(len(par), par.ctypes.data)
        opt = _lib.rsd_options(mode, prec_leaf, prec_mid, prec_root, maxit,
                               _stream() if torch.cuda.is_available() else 0, int(profile), wait_cycles,
                               gamma, krylov, restart, tune_cache.encode() if tune_cache else None,
                               int(nonsymmetric))
        out = C.c_void_p()
        rc = lib.rsd_setup(C.byref(csr), _ptr(dof_node), C.byref(tree), C.byref(opt), C.byref(out))
        if rc != 0:
            if out.value:
                lib.rsd_destroy(out)
            raise RSDError(rc, "rsd_setup")
        return cls(out.value, n)

    @classmethod
    def setup_batched(cls, problems, prec_leaf: int = RSD_PREC_TF32, prec_mid: int = RSD_PREC_TF32,
                      prec_root: int = RSD_PREC_FP64, maxit: int = 200, profile: bool = False,
                      tune_cache: str | None = None) -> "RSD":
        """One hierarchy for several independent problems (dicts with rowptr, col, val,
        dof_node, parent, all on the device).  Vectors are the problems' concatenation."""
        lib = _lib.load()
        n = len(problems)
        keep = []
        csrs = (_lib.rsd_csr * n)()
        trees = (_lib.rsd_tree * n)()
        owners = (C.c_void_p * n)()
        total = 0
        for i, pr in enumerate(problems):
            rp = pr["rowptr"].to(torch.int64).contiguous()
            cl = pr["col"].to(torch.int32).contiguous()
            vl = pr["val"].to(torch.float64).contiguous()
            ow = pr["dof_node"].to(torch.int32).contiguous()
            par = np.ascontiguousarray(np.asarray(pr["parent"], dtype=np.int32))
            keep += [rp, cl, vl, ow, par]
            csrs[i] = _lib.rsd_csr(rp.numel() - 1, cl.numel(), _ptr(rp), _ptr(cl), _ptr(vl),
                                   RSD_MEM_DEVICE if rp.is_cuda else RSD_MEM_HOST)
            trees[i] = _lib.rsd_tree(len(par), par.ctypes.data)
            owners[i] = _ptr(ow)
            total += rp.numel() - 1
        opt = _lib.rsd_options(RSD_MODE_EXACT, prec_leaf, prec_mid, prec_root, maxit,
                               _stream() if torch.cuda.is_available() else 0, int(profile), 0, 0, 0, 0,
                               tune_cache.encode() if tune_cache else None)
        out = C.c_void_p()
        rc = lib.rsd_setup_batched(n, csrs, owners, trees, C.byref(opt), C.byref(out))
        del keep
        if rc != 0:
            if out.value:
                lib.rsd_destroy(out)
            raise RSDError(rc, "rsd_setup_batched")
        return cls(out.value, total)

    def __del__(self):
        try:
            if self._h and self._h.value:
                _lib.load().rsd_destroy(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    close = __del__

    def apply(self, r: torch.Tensor, z: torch.Tensor | None = None) -> torch.Tensor:
        z = torch.empty_like(r) if z is None else z
        check(_lib.load().rsd_apply(self._h, _ptr(r), _ptr(z)), "rsd_apply")
        return z

    def solve(self, f: torch.Tensor, tol: float = 1e-8, u: torch.Tensor | None = None,
              allow_noconv: bool = False):
        u = torch.empty_like(f) if u is None else u
        st = _lib.rsd_stats()
        rc = _lib.load().rsd_solve(self._h, _ptr(f), _ptr(u), tol, C.byref(st))
        if rc != 0 and not (allow_noconv and rc == _lib.RSD_ERR_NOCONV):
            raise RSDError(rc, "rsd_solve")
        hist = [st.history[i] for i in range(min(st.iterations + 1, 64))]
        return u, dict(iterations=st.iterations, relres=st.relres,
                       relres_recursive=st.relres_recursive, history=hist)

    def solve_adjoint(self, g: torch.Tensor, tol: float = 1e-8, lam: torch.Tensor | None = None,
                      allow_noconv: bool = False):
        """lam with K^T lam = g on the same hierarchy (rsd_solve_adjoint)."""
        lam = torch.empty_like(g) if lam is None else lam
        st = _lib.rsd_stats()
        rc = _lib.load().rsd_solve_adjoint(self._h, _ptr(g), _ptr(lam), tol, C.byref(st))
        if rc != 0 and not (allow_noconv and rc == _lib.RSD_ERR_NOCONV):
            raise RSDError(rc, "rsd_solve_adjoint")
        return lam, dict(iterations=st.iterations, relres=st.relres)

    def check(self) -> None:
        check(_lib.load().rsd_check(self._h), "rsd_check")

    def profile(self, reset: bool = True) -> dict:
        """Per kernel class: launches, device ms (CUDA events), algorithmic flops and bytes."""
        p = _lib.rsd_profile_t()
        check(_lib.load().rsd_profile(self._h, C.byref(p), int(reset)), "rsd_profile")
        out = {name: dict(launches=p.launches[i], ms=p.ms[i], flops=p.flops[i], bytes=p.bytes[i])
               for i, name in enumerate(_lib.PROFILE_CLASSES)}
        out["host_analysis_ms"] = p.host_analysis_ms
        out["host_parts_ms"] = dict(zip(["copy", "sort", "check", "sets", "maps", "plan"], list(p.host_parts_ms)))
        out["host_issue_ms"] = p.host_issue_ms
        return out

    def trace(self) -> list[dict]:
        """Per-launch profile records (class, stream, start/end ms, flops, bytes) in issue
        order; call before a resetting profile()."""
        lib = _lib.load()
        n = C.c_int64()
        check(lib.rsd_profile_trace(self._h, None, 0, C.byref(n)), "rsd_profile_trace")
        recs = (_lib.rsd_trace_rec * max(n.value, 1))()
        check(lib.rsd_profile_trace(self._h, recs, n.value, C.byref(n)), "rsd_profile_trace")
        return [dict(cls=_lib.PROFILE_CLASSES[r.cls], stream=r.stream, start_ms=r.start_ms, end_ms=r.end_ms,
                     flops=r.flops, bytes=r.bytes, issue_ms=r.issue_ms) for r in recs[: n.value]]

    def info(self) -> dict:
        inf = _lib.rsd_info_t()
        check(_lib.load().rsd_get_info(self._h, C.byref(inf)), "rsd_get_info")
        return {k: getattr(inf, k) for k, _ in _lib.rsd_info_t._fields_}

    def front_dims(self, node: int) -> tuple[int, int, int]:
        s, b, lv = C.c_int32(), C.c_int32(), C.c_int32()
        check(_lib.load().rsd_front_dims(self._h, node, C.byref(s), C.byref(b), C.byref(lv)), "rsd_front_dims")
        return s.value, b.value, lv.value

    def front_dofs(self, node: int) -> np.ndarray:
        s, b, _ = self.front_dims(node)
        out = np.empty(s + b, dtype=np.int32)
        check(_lib.load().rsd_front_dofs(self._h, node, out.ctypes.data), "rsd_front_dofs")
        return out

    def front_map(self, node: int) -> np.ndarray:
        _, b, _ = self.front_dims(node)
        out = np.empty(max(b, 1), dtype=np.int32)
        check(_lib.load().rsd_front_map(self._h, node, out.ctypes.data), "rsd_front_map")
        return out[:b]

    def front_factor(self, node: int) -> np.ndarray:
        s, b, _ = self.front_dims(node)
        out = np.empty((s + b) * max(s, 1), dtype=np.float64)
        check(_lib.load().rsd_front_factor(self._h, node, out.ctypes.data), "rsd_front_factor")
        return out[: (s + b) * s].reshape(s + b, s)

    def front_factor_upper(self, node: int) -> np.ndarray:
        """Nonsymmetric fronts: [U^T; Y^T] (rsd_front_factor_upper)."""
        s, b, _ = self.front_dims(node)
        out = np.empty((s + b) * max(s, 1), dtype=np.float64)
        check(_lib.load().rsd_front_factor_upper(self._h, node, out.ctypes.data), "rsd_front_factor_upper")
        return out[: (s + b) * s].reshape(s + b, s)

    def front_factor16(self, node: int) -> np.ndarray:
        """The FP16 factor copy a TF32 level's sweeps read, unscaled (rsd_front_factor16)."""
        s, b, _ = self.front_dims(node)
        out = np.empty((s + b) * max(s, 1), dtype=np.float64)
        check(_lib.load().rsd_front_factor16(self._h, node, out.ctypes.data), "rsd_front_factor16")
        return out[: (s + b) * s].reshape(s + b, s)


    def front_dinv(self, node: int) -> np.ndarray:
        """The inverted 128 x 128 diagonal blocks the sweeps apply, shape (nd, 128, 128)
        (rsd_front_dinv)."""
        s, _, _ = self.front_dims(node)
        nd = (s + 127) // 128
        out = np.empty(max(nd, 1) * 128 * 128, dtype=np.float64)
        check(_lib.load().rsd_front_dinv(self._h, node, out.ctypes.data), "rsd_front_dinv")
        return out[: nd * 128 * 128].reshape(nd, 128, 128)

class DiffusionSolve(torch.autograd.Function):
    """u = K(exp(m))^-1 b for -div(kappa grad u) = f on the n^3 grid, differentiable in the
    per-element log-coefficient m and the load b.  Forward: rsd_grid_exp, rsd_grid_assemble,
    rsd_setup, rsd_solve.  Backward (the adjoint method): lam = rsd_solve_adjoint(dL/du) on
    the forward's hierarchy, dL/dm = rsd_grid_coef_grad(u, lam, kappa), dL/db = lam."""

    @staticmethod
    def forward(ctx, m, b, n, depth, tol, precs, maxit):
        kappa = grid_exp(n, m.detach())
        prob = _grid_system(n, depth, kappa)
        h = RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                      prec_leaf=precs[0], prec_mid=precs[1], prec_root=precs[2], maxit=maxit)
        u, st = h.solve(b.detach().to(torch.float64).contiguous(), tol=tol)
        ctx.h, ctx.n, ctx.tol, ctx.stats = h, n, tol, st
        ctx.save_for_backward(kappa, u)
        return u

    @staticmethod
    def backward(ctx, gu):
        kappa, u = ctx.saved_tensors
        lam, _ = ctx.h.solve_adjoint(gu.to(torch.float64).contiguous(), tol=ctx.tol)
        _, dm = coef_grad(ctx.n, u, lam, kappa)
        return dm, lam, None, None, None, None, None


def diffusion_solve(m: torch.Tensor, b: torch.Tensor, n: int, depth: int, tol: float = 1e-10,
                    precs=(RSD_PREC_FP64, RSD_PREC_FP64, RSD_PREC_FP64), maxit: int = 500) -> torch.Tensor:
    """Differentiable solve (DiffusionSolve.apply); m: (n-1)^3 elements, b: (n-2)^3 nodes."""
    return DiffusionSolve.apply(m, b, n, depth, tol, tuple(precs), maxit)
