"""User-facing wrappers: a factorization object and the autograd function.

`Factorization` owns the tree and factor handles of libfmmlu; its `solve` and
`solve_adjoint` apply A^{-1} and A^{-H} with the factors resident in device
memory. `FMMLUSolve` is a torch.autograd.Function whose forward is
fmmlu_solve and whose backward applies the adjoint factors (fmmlu_solve_adjoint),
following torch's convention for complex gradients: for x = A^{-1} b and a
real loss L, grad_b = A^{-H} grad_x.
"""
from __future__ import annotations

import math

import torch

from . import binding as B


def _as_cuda(t, dtype, device):
    t = torch.as_tensor(t)
    if t.device.type != "cuda":
        t = t.to(dtype).pin_memory().to(device, non_blocking=True) if t.device.type == "cpu" \
            else t.to(device)
    return t.to(dtype).contiguous()


class Factorization:
    """FMM-LU factorization of the sqrt(w)-scaled CFIE system on one GPU."""

    def __init__(self, points, normals, weights, k: float, eps: float, eta: float | None = None,
                 leaf_size: int = 64, n_proxy: int = 300, proxy_radius_factor: float = 1.5,
                 precision: int = B.PRECISION_AUTO, verbose: int = 0, device=None,
                 **extra_opts):
        device = torch.device(device or "cuda")
        self.device = device
        self.points = _as_cuda(points, torch.float64, device)
        self.normals = _as_cuda(normals, torch.float64, device)
        self.weights = _as_cuda(weights, torch.float64, device)
        self.n = int(self.points.shape[0])
        self.k = float(k)
        self.eta = float(k) if eta is None else float(eta)
        self.eps = float(eps)
        self.opts = B.fmmlu_default_opts(
            leaf_size=leaf_size, eta=self.eta if eta is not None else math.nan,
            n_proxy=n_proxy, proxy_radius_factor=proxy_radius_factor, precision=precision,
            verbose=verbose, **extra_opts)
        self.tree = None
        self.handle = None
        self.tree = B.fmmlu_build_tree(self.points, self.opts)
        self.handle = B.fmmlu_factor(self.tree, self.points, self.normals, self.weights,
                                     self.k, self.eps, self.opts)

    def _vec(self, b):
        b = _as_cuda(b, torch.complex128, self.device)
        if b.dim() == 2 and b.shape[0] == self.n and b.shape[1] != self.n:
            return b.t().contiguous(), True       # (n, nrhs) -> (nrhs, n)
        return b, False

    def solve(self, b):
        """x = A^{-1} b; b is (n,) or (n, nrhs) (any device); returns CUDA."""
        bb, tr = self._vec(b)
        x = torch.empty_like(bb)
        B.fmmlu_solve(self.handle, bb, x, self.n)
        return x.t() if tr else x

    def solve_adjoint(self, b):
        bb, tr = self._vec(b)
        x = torch.empty_like(bb)
        B.fmmlu_solve_adjoint(self.handle, bb, x, self.n)
        return x.t() if tr else x

    def gmres(self, b, tol: float = 1e-10, restart: int = 30, maxiter: int = 200):
        """x with A x = b by GMRES preconditioned by this factorization (Sec. 7);
        returns (x, iters, relres, converged)."""
        bb, tr = self._vec(b)
        x = torch.empty_like(bb)
        its, rel, ok = B.fmmlu_gmres(self.handle, self.points, self.normals, self.weights, bb, x,
                                     self.n, tol, restart, maxiter)
        return (x.t() if tr else x), its, rel, ok

    def sonar_cross_section(self, phis, batch: int = 64):
        """Monostatic backscattered far field R(phi) for incident plane waves
        along d = (cos phi, sin phi, 0) (Sec. 6.3); returns complex128 (m,)."""
        ph = torch.as_tensor(phis, dtype=torch.float64)
        dirs = torch.stack([torch.cos(ph), torch.sin(ph), torch.zeros_like(ph)], dim=1)
        dirs = dirs.to(self.device).contiguous()
        R = torch.empty(dirs.shape[0], dtype=torch.complex128, device=self.device)
        B.fmmlu_sonar_sweep(self.handle, self.points, self.normals, self.weights, dirs, R, batch)
        return R

    def matvec(self, v):
        """A v by the dense on-the-fly product (independent of the factors)."""
        vv, tr = self._vec(v)
        y = torch.empty_like(vv)
        B.fmmlu_matvec(self.points, self.normals, self.weights, self.k, self.eta, vv, y)
        return y.t() if tr else y

    def stats(self) -> dict:
        return B.fmmlu_stats(self.handle)

    def free(self):
        if self.handle is not None:
            B.fmmlu_free(self.handle)
            self.handle = None
        if self.tree is not None:
            B.fmmlu_free(self.tree)
            self.tree = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class FMMLUSolve(torch.autograd.Function):
    """x = A^{-1} b with gradient grad_b = A^{-H} grad_x (factors reused)."""

    @staticmethod
    def forward(ctx, b, fac: Factorization):
        ctx.fac = fac
        return fac.solve(b).contiguous()

    @staticmethod
    def backward(ctx, grad_x):
        return ctx.fac.solve_adjoint(grad_x.contiguous()), None


def fmmlu_solve_autograd(fac: Factorization, b: torch.Tensor) -> torch.Tensor:
    return FMMLUSolve.apply(b, fac)
