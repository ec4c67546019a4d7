"""PyTorch autograd around the C ABI's 2D adjoint.

`HwenoRun2D(cfg)(u0, nsteps, checkpoint_every)` returns the state after nsteps
Runge-Kutta steps of the 2D hybrid HWENO scheme (Zhao & Qiu,
arXiv:2002.08816, Sec. 2.2) from the moments u0 ([C][3][ny][nx], a CUDA
tensor in the configured precision), and its backward is hweno_backward: the
vector-Jacobian product with the troubled cells, the Lax-Friedrichs speeds and
the time steps of the forward run held fixed, recomputing each checkpoint
segment.  Argument marshalling only: every step runs in libhweno's kernels.
The handle is bound to the CUDA stream current when the object is made.
"""

import torch

from . import hweno as H


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, handle, precision, nsteps, checkpoint_every, t_final):
        u0 = u0.contiguous()
        H.hweno_set_state(handle, u0.data_ptr(), precision, True)
        H.hweno_record(handle, nsteps, checkpoint_every, t_final)
        out = torch.empty_like(u0)
        H.hweno_get_state(handle, out.data_ptr(), precision, True)
        ctx.handle = handle
        ctx.precision = precision
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.contiguous()
        grad_in = torch.empty_like(g)
        H.hweno_backward(ctx.handle, g.data_ptr(), grad_in.data_ptr(), ctx.precision, True)
        return grad_in, None, None, None, None, None


class HwenoRun2D:
    """A 2D periodic configuration (hweno.make_config) with a device handle;
    call it on initial moments to get the final ones, differentiably."""

    def __init__(self, cfg):
        if cfg.dim != 2 or cfg.bc != H.HWENO_BC_PERIODIC:
            raise ValueError("HwenoRun2D needs a 2D periodic configuration")
        self.cfg = cfg
        self.dtype = torch.float64 if cfg.precision == H.HWENO_FP64 else torch.float32
        self.handle = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)

    def __call__(self, u0, nsteps, checkpoint_every=20, t_final=-1.0):
        if u0.dtype != self.dtype or not u0.is_cuda:
            raise TypeError("u0 must be a CUDA tensor of %s" % self.dtype)
        return _Run.apply(u0, self.handle, self.cfg.precision, int(nsteps), int(checkpoint_every),
                          float(t_final))

    def close(self):
        if self.handle:
            H.hweno_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
