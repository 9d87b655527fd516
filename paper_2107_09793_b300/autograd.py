"""torch.autograd.Function over jet_contract / jet_contract_grad.

Forward: the values of the chosen input tensors are copied into the network
(jet_tensor_update) and the amplitudes are contracted on the GPU.  Backward:
torch hands over g_b = dL/d conj(amp_b) (conjugate Wirtinger convention); the
amplitude is holomorphic in every tensor, so dL/d conj(G) = conj(sum_b conj(g_b)
d amp_b / dG) = conj(env_G) with cot_b = conj(g_b), which jet_contract_grad
returns (adjoint sweep, per-slice recomputation).  Argument marshalling only.
"""
import numpy as np
import torch


class Amplitudes(torch.autograd.Function):
    @staticmethod
    def forward(ctx, net, outputs, tensor_ids, *tensors):
        for tid, t in zip(tensor_ids, tensors):
            net.update(int(tid), t.detach().to("cpu", torch.complex64).numpy())
        amps = net.contract(outputs)
        ctx.net, ctx.outputs, ctx.ids = net, np.asarray(outputs), list(tensor_ids)
        ctx.dtypes = [(t.dtype, t.device) for t in tensors]
        return torch.from_numpy(amps).to(tensors[0].device if tensors else "cpu")

    @staticmethod
    def backward(ctx, grad_amps):
        cot = np.conj(grad_amps.detach().to("cpu", torch.complex128).numpy())
        _, envs = ctx.net.contract_grad(ctx.outputs, cot, ctx.ids)
        grads = [torch.from_numpy(np.conj(e)).to(device=dev, dtype=dt) for e, (dt, dev) in zip(envs, ctx.dtypes)]
        return (None, None, None, *grads)


def amplitudes(net, outputs, tensor_ids, tensors):
    """Differentiable amplitudes of `outputs` with respect to `tensors` (values of tensor_ids)."""
    return Amplitudes.apply(net, outputs, list(tensor_ids), *tensors)
