"""Differentiable GraphGP operations (torch.autograd.Function over the C ABI).

theta is a float64 tensor [lengthscale, sigma2, nugget] of the stationary
covariance of Sec. 2.1; gradients with respect to it come from the library's
adjoint kernels (Sec. 2.3: derivatives through the Cholesky factors, which are
recomputed rather than stored).  Vectors are float32 CUDA tensors in graph
order.  Every function builds the factor for the given theta (one
graphgp_factor call) unless a Factor is passed in.

    v   = generate(graph, kernel_type, theta, xi)      # v = L xi
    xi  = whiten(graph, kernel_type, theta, v)         # xi = L^-1 v
    ld  = logdet(graph, kernel_type, theta)            # log det L L^T
    nll = nll(graph, kernel_type, theta, v)            # 0.5 xi.xi + 0.5 ld
    nll = nll(graph, kernel_type, theta, v, points)    # also d/d points
    nll = nll_fit(graph, kernel_type, theta, v)        # one pass (k <= 32)

With `points` (the [N, d] tensor the graph was built from; its values are
not read again) the NLL is also differentiable with respect to the point
coordinates, the graph (order, neighbour lists, levels) held fixed.
"""
from __future__ import annotations

import torch

from . import (Factor, Graph, Kernel, factor as _factor, generate_backward, logdet as _logdet,
               nll as _nll, nll_backward, nll_backward_points, nll_grad_fused, whiten_backward,
               generate as _generate, whiten as _whiten)


def _kernel(kernel_type: int, theta: torch.Tensor) -> Kernel:
    t = theta.detach().double().cpu()
    return Kernel(int(kernel_type), float(t[1]), float(t[0]), float(t[2]))


def _theta_grad(tb, theta: torch.Tensor):
    return None if tb is None else tb.to(device=theta.device, dtype=theta.dtype)


class _Generate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi, theta, graph, kernel_type):
        f = _factor(graph, _kernel(kernel_type, theta))
        v = _generate(graph, f, xi.contiguous())
        ctx.graph, ctx.fac = graph, f
        ctx.save_for_backward(xi, v, theta)
        return v

    @staticmethod
    def backward(ctx, grad_v):
        xi, v, theta = ctx.saved_tensors
        xibar, tb = generate_backward(ctx.graph, ctx.fac, xi.contiguous(), v,
                                      grad_v.contiguous().float(),
                                      theta=ctx.needs_input_grad[1])
        return xibar, _theta_grad(tb, theta), None, None


class _Whiten(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, theta, graph, kernel_type):
        f = _factor(graph, _kernel(kernel_type, theta))
        xi = _whiten(graph, f, v.contiguous())
        ctx.graph, ctx.fac = graph, f
        ctx.save_for_backward(v, xi, theta)
        return xi

    @staticmethod
    def backward(ctx, grad_xi):
        v, xi, theta = ctx.saved_tensors
        vbar, tb = whiten_backward(ctx.graph, ctx.fac, v.contiguous(), xi,
                                   grad_xi.contiguous().float(), 0.0,
                                   theta=ctx.needs_input_grad[1])
        return vbar, _theta_grad(tb, theta), None, None


class _Logdet(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, graph, kernel_type):
        f = _factor(graph, _kernel(kernel_type, theta))
        ctx.graph, ctx.fac = graph, f
        ctx.save_for_backward(theta)
        return _logdet(f).reshape(())

    @staticmethod
    def backward(ctx, grad):
        (theta,) = ctx.saved_tensors
        g = ctx.graph
        z = torch.zeros(g.N, dtype=torch.float32, device="cuda")
        _, tb = whiten_backward(g, ctx.fac, z, z, z, float(grad.item()))
        return _theta_grad(tb, theta), None, None


class _Nll(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, theta, graph, kernel_type):
        f = _factor(graph, _kernel(kernel_type, theta))
        out = _nll(graph, f, v.contiguous()).reshape(())
        ctx.graph, ctx.fac = graph, f
        ctx.save_for_backward(v, theta)
        return out

    @staticmethod
    def backward(ctx, grad):
        v, theta = ctx.saved_tensors
        vbar, tb = nll_backward(ctx.graph, ctx.fac, v.contiguous(), float(grad.item()),
                                theta=ctx.needs_input_grad[1])
        return vbar, _theta_grad(tb, theta), None, None


class _NllPoints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, theta, points, graph, kernel_type):
        f = _factor(graph, _kernel(kernel_type, theta))
        out = _nll(graph, f, v.contiguous()).reshape(())
        ctx.graph, ctx.fac = graph, f
        ctx.save_for_backward(v, theta, points)
        return out

    @staticmethod
    def backward(ctx, grad):
        v, theta, points = ctx.saved_tensors
        g = float(grad.item())
        vbar, tb = nll_backward(ctx.graph, ctx.fac, v.contiguous(), g,
                                theta=ctx.needs_input_grad[1])
        pbar = None
        if ctx.needs_input_grad[2]:
            d = points.shape[1]
            pbar = nll_backward_points(ctx.graph, ctx.fac, v.contiguous(), g)[:, :d]
            pbar = pbar.to(device=points.device, dtype=points.dtype)
        return vbar, _theta_grad(tb, theta), pbar, None, None


class _NllFit(torch.autograd.Function):
    """The NLL of a fit step: value and gradient come from one pass with the
    factors recomputed (graphgp_nll_grad_fused), so backward only scales the
    stored gradient by the incoming cotangent."""

    @staticmethod
    def forward(ctx, v, theta, graph, kernel_type):
        out, vbar, tb = nll_grad_fused(graph, _kernel(kernel_type, theta), v.contiguous())
        ctx.save_for_backward(vbar, _theta_grad(tb, theta))
        return out.reshape(())

    @staticmethod
    def backward(ctx, grad):
        vbar, tb = ctx.saved_tensors
        return (vbar * grad.to(device=vbar.device, dtype=vbar.dtype),
                tb * grad.to(device=tb.device, dtype=tb.dtype), None, None)


def generate(graph: Graph, kernel_type: int, theta: torch.Tensor, xi: torch.Tensor):
    return _Generate.apply(xi, theta, graph, kernel_type)


def whiten(graph: Graph, kernel_type: int, theta: torch.Tensor, v: torch.Tensor):
    return _Whiten.apply(v, theta, graph, kernel_type)


def logdet(graph: Graph, kernel_type: int, theta: torch.Tensor):
    return _Logdet.apply(theta, graph, kernel_type)


def nll(graph: Graph, kernel_type: int, theta: torch.Tensor, v: torch.Tensor,
        points: torch.Tensor | None = None):
    if points is None:
        return _Nll.apply(v, theta, graph, kernel_type)
    if points.shape != (graph.N, points.shape[1]) or not 1 <= points.shape[1] <= 3:
        raise ValueError("points must be the [N, d] tensor the graph was built from")
    return _NllPoints.apply(v, theta, points, graph, kernel_type)


def nll_fit(graph: Graph, kernel_type: int, theta: torch.Tensor, v: torch.Tensor):
    """nll() for a fit (k <= 32): the gradient with respect to v and theta is
    computed in the same pass as the value, each conditional once."""
    return _NllFit.apply(v, theta, graph, kernel_type)
