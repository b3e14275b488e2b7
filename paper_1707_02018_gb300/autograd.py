"""Autograd wrappers: W and W^*, R and R^* as each other's backward.

The backward of a linear operator is its adjoint, so the exact W^* of Eq. 4
(not W^dagger) is what makes d/dc of a loss through W correct; likewise R^*
for R.  Each Function calls the library's kernels in both directions (the
plan objects carry the operator); tensors use the library layouts (images
rows x image_pitch, coefficient vectors in the padded packed order).
"""
import torch

from . import blur, blur_adjoint, wt_synth, wt_synth_adjoint


class WtSynth(torch.autograd.Function):
    """image = W coeffs; backward: grad_coeffs = W^* grad_image."""

    @staticmethod
    def forward(ctx, coeffs, plan):
        ctx.plan = plan
        return wt_synth(plan, coeffs.contiguous())

    @staticmethod
    def backward(ctx, grad_image):
        return wt_synth_adjoint(ctx.plan, grad_image.contiguous()), None


class WtSynthAdjoint(torch.autograd.Function):
    """coeffs = W^* image; backward: grad_image = W grad_coeffs."""

    @staticmethod
    def forward(ctx, image, plan):
        ctx.plan = plan
        return wt_synth_adjoint(plan, image.contiguous())

    @staticmethod
    def backward(ctx, grad_coeffs):
        return wt_synth(ctx.plan, grad_coeffs.contiguous()), None


class Blur(torch.autograd.Function):
    """out = R x; backward: grad_x = R^* grad_out."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return blur(plan, x.contiguous())

    @staticmethod
    def backward(ctx, grad_out):
        return blur_adjoint(ctx.plan, grad_out.contiguous()), None


class BlurAdjoint(torch.autograd.Function):
    """out = R^* x; backward: grad_x = R grad_out."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return blur_adjoint(plan, x.contiguous())

    @staticmethod
    def backward(ctx, grad_out):
        return blur(ctx.plan, grad_out.contiguous()), None


def synth(coeffs, plan):
    return WtSynth.apply(coeffs, plan)


def synth_adjoint(image, plan):
    return WtSynthAdjoint.apply(image, plan)


def apply_blur(x, plan):
    return Blur.apply(x, plan)


def apply_blur_adjoint(x, plan):
    return BlurAdjoint.apply(x, plan)
