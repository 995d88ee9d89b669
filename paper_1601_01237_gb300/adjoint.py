"""Differentiable rollout: torch.autograd.Function over the C ABI's
lbm_record (forward with checkpoints) and lbm_adjoint (hand-written reverse
pass).  Torch only carries tensors and the stream; the forward steps and the
reverse steps run in the CUDA library."""
import torch

from .lattice import Lattice


class LBMRollout(torch.autograd.Function):
    """rho1_N, rho2_N = LBMRollout.apply(rho1_0, rho2_0, G12, tau1, shape, n_steps,
    ckpt_every, options)

    rho1_0, rho2_0: CUDA float64 tensors of shape (nz, ny, nx), the initial
    densities (the run starts at rest, f = w_i rho).  G12: 0-d tensor, the
    signed G^{12} = G^{21} of Eq. 7 (tied).  tau1: 0-d tensor.  options: dict of
    further Lattice arguments (tau2, storage, g_ext, periodic, collision, ...).
    Gradients flow to rho1_0, rho2_0, G12 and tau1."""

    @staticmethod
    def forward(ctx, rho1_0, rho2_0, G12, tau1, shape, n_steps, ckpt_every, options):
        opts = dict(options)
        tau2 = opts.pop("tau2", float(tau1))
        lat = Lattice(shape, tau=(float(tau1), float(tau2)), G12=float(G12), G21=float(G12),
                      stream=torch.cuda.current_stream().cuda_stream, **opts)
        lat.init_fields(rho1_0.detach().double().contiguous(), rho2_0.detach().double().contiguous())
        lat.record(n_steps, ckpt_every)
        r1 = torch.empty(shape, dtype=torch.float64, device=rho1_0.device)
        r2 = torch.empty(shape, dtype=torch.float64, device=rho1_0.device)
        lat.moments_device(rho1=r1, rho2=r2, out_f64=True)
        ctx.lat = lat
        return r1, r2

    @staticmethod
    def backward(ctx, g1, g2):
        lat = ctx.lat
        shape = lat.shape
        dev = g1.device if g1 is not None else g2.device
        d1 = torch.empty(shape, dtype=torch.float64, device=dev)
        d2 = torch.empty(shape, dtype=torch.float64, device=dev)
        par = lat.adjoint(None if g1 is None else g1.double().contiguous(),
                          None if g2 is None else g2.double().contiguous(), d1, d2)
        lat.close()
        ctx.lat = None
        dG = torch.tensor(par[0] + par[1], dtype=torch.float64, device=dev)
        dtau1 = torch.tensor(par[2], dtype=torch.float64, device=dev)
        return d1, d2, dG, dtau1, None, None, None, None
