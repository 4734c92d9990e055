"""torch.autograd access to the bucket-domain refinement loss (rsft_refine_eval).

``BucketResidual.apply(freq, amp_ri, plan)`` returns the loss
E = sum_l ||F_l - fold_l(s_theta)||^2 of K tones (freq: float32 [K, D] cycles/sample,
amp_ri: float32 [K, 2] real and imaginary parts, both on the plan's device) against the
buckets of the plan's last ``rsft_refine_prepare`` or execute.  The forward pass runs the
library's kernels and keeps their gradient; the backward pass scales it.  Only argument
marshalling happens here.
"""
import torch

from . import rsft_refine_eval


class BucketResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, freq, amp_ri, plan):
        freq_c = freq.detach().contiguous().to(torch.float32)
        amp_c = torch.view_as_complex(amp_ri.detach().to(torch.float32).contiguous())
        loss = torch.zeros(1, dtype=torch.float64, device=freq.device)
        gf = torch.empty_like(freq_c)
        ga = torch.empty_like(amp_c)
        rsft_refine_eval(plan, freq_c, amp_c, loss=loss, grad_freq=gf, grad_amp=ga)
        ctx.save_for_backward(gf, torch.view_as_real(ga))
        return loss[0].to(freq.dtype)

    @staticmethod
    def backward(ctx, gout):
        gf, ga = ctx.saved_tensors
        return gout * gf, gout * ga, None
