"""torch.autograd.Function over the scan log-likelihood (argument marshalling only).

ScanLogLik.apply(xi, filt, scan) returns ll[P], the log-likelihood of the scan
for every particle of `filt` at the pose T0 exp(xi_i) (T0: the particle's current
pose, neighbour keyframes as last selected). The forward runs the value-only
lookup pass; the backward runs the lookup pass with gradient at the same poses
and the chain rule through the SE(3) right Jacobian, both in CUDA
(gmcs_loglik / gmcs_loglik_backward).

The backward reads T0 and the neighbour sets from the filter again, so it is
only the derivative of the forward if the filter has not changed in between: the
forward records the filter's state version (gmcs_state_version) and the backward
raises if any call since (a step, a move, a new selection or keyframe, ...)
has changed it.
"""
import torch


class ScanLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi, filt, scan):
        if not (xi.is_cuda and scan.is_cuda):
            raise ValueError("xi and scan must be CUDA tensors")
        xi = xi.detach().to(torch.float32).contiguous()
        scan = scan.detach().to(torch.float32).contiguous()
        ll = torch.empty(xi.shape[0], dtype=torch.float32, device=xi.device)
        filt.loglik(xi, scan, ll)
        ctx.filt = filt
        ctx.version = filt.state_version()
        ctx.save_for_backward(xi, scan)
        return ll

    @staticmethod
    def backward(ctx, grad_ll):
        xi, scan = ctx.saved_tensors
        if ctx.filt.state_version() != ctx.version:
            raise RuntimeError("ScanLogLik backward: the filter's poses, neighbours or keyframes changed since the "
                               "forward (state version %d -> %d); run the forward again"
                               % (ctx.version, ctx.filt.state_version()))
        grad_xi = torch.empty_like(xi)
        ctx.filt.loglik_backward(xi, scan, grad_ll.detach().to(torch.float32).contiguous(), grad_xi)
        return grad_xi, None, None


def scan_loglik(xi, filt, scan):
    return ScanLogLik.apply(xi, filt, scan)
