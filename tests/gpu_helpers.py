"""Shared plumbing for the GPU parity tests: build/load the C-ABI library
and run a workloads.Problem through it (argument marshalling only)."""
from __future__ import annotations

import numpy as np


def lib():
    from paper_2311_05595_gb300 import build as b

    b.build()
    from paper_2311_05595_gb300 import tosolve as T

    return T


def desc_for(T, p, precision, levels=None, max_rhs=None, **extra):
    """extra: further descriptor fields (smoother, cheb_degree, inner_its)."""
    return T.make_desc(p.nx, p.ny, p.nz, degree=p.degree, n_mr=p.n_mr, d_mr=getattr(p, "d_mr", None),
                       E0=p.E0, Emin=p.Emin, nu=p.nu,
                       penal=p.penal, rmin=p.rmin, mg_levels=levels or p.mg_levels,
                       precision=precision, max_rhs=max_rhs or p.nrhs,
                       family=1 if getattr(p, "family", "lagrange") == "serendipity" else 0, **extra)


class Run:
    """A problem set up on the GPU: handle, stream, device copies of x and f."""

    def __init__(self, p, precision, levels=None, max_rhs=None, **extra):
        import torch

        self.T = T = lib()
        self.torch = torch
        self.p = p
        self.dev = torch.device("cuda:0")
        self.stream = torch.cuda.Stream()
        self.solver = T.Solver(desc_for(T, p, precision, levels, max_rhs, **extra), p.mask, self.stream,
                               elem_q1=getattr(p, "elem_q1", None))
        self.h = self.solver.h
        self.x = torch.tensor(p.x, device=self.dev)
        f = np.array(p.f, dtype=np.float64)
        self.f = torch.tensor(f, device=self.dev)

    def set_densities(self, x=None):
        with self.torch.cuda.stream(self.stream):
            self.T.tosolve_set_densities(self.h, self.x if x is None else x)
        self.stream.synchronize()

    def solve(self, rtol=1e-8, maxit=2000, u0=None, nrhs=None, raise_on_error=True):
        nrhs = nrhs or self.p.nrhs
        u = self.torch.zeros((nrhs, self.p.ndof), dtype=self.torch.float64, device=self.dev) \
            if u0 is None else u0.clone()
        with self.torch.cuda.stream(self.stream):
            info = self.T.tosolve_solve(self.h, self.f[:nrhs].contiguous(), nrhs, u, rtol, maxit,
                                        raise_on_error=raise_on_error)
        self.stream.synchronize()
        return u, info

    def grad(self, u, nrhs=None):
        nrhs = nrhs or self.p.nrhs
        gx = self.torch.zeros_like(self.x)
        gr = self.torch.zeros_like(self.x)
        with self.torch.cuda.stream(self.stream):
            c = self.T.tosolve_compliance_grad(self.h, u, self.f[:nrhs].contiguous(), nrhs, gx, gr)
        self.stream.synchronize()
        return c, gx.cpu().numpy(), gr.cpu().numpy()

    def apply(self, level, precision, x):
        import torch

        xd = torch.tensor(x, device=self.dev)
        y = torch.zeros_like(xd)
        with torch.cuda.stream(self.stream):
            self.T.tosolve_apply(self.h, level, precision, xd, y)
        self.stream.synchronize()
        return y.cpu().numpy()

    def precondition(self, b):
        import torch

        bd = torch.tensor(b, device=self.dev)
        z = torch.zeros_like(bd)
        with torch.cuda.stream(self.stream):
            self.T.tosolve_precondition(self.h, bd, z)
        self.stream.synchronize()
        return z.cpu().numpy()

    def close(self):
        self.solver.close()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))
