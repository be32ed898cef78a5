"""CNN_skel: the generator of the canonical weight volume (oracle, FP64, PyTorch CPU ops).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

Sec. 4.2 generates the weight volume W^c from a constant random latent z with a
CNN; the network's figure caption fixes its shape: a fully-connected layer, a
reshape, and five 3D transposed convolutions in sequence, z of size 256 in,
a 32 x 32 x 32 x 25 volume out.  Readings (the paper prints no more):
  * the fully-connected layer maps z to C0 values, read as a C0 x 1 x 1 x 1 tensor;
  * each transposed convolution has kernel 4, stride 2 and padding 1, so five of
    them take 1^3 to 32^3; channels C0 -> C1 -> C2 -> C3 -> C4 -> 25;
  * LeakyReLU with slope 0.2 after the fully-connected layer and after every
    transposed convolution but the last;
  * the 25 output channels (24 bones + background) pass through a softmax over
    channels, after adding log(prior) when a prior volume is given, so that the
    weights at a voxel form a partition of unity.
The transposed convolution is the library routine (torch conv_transpose3d,
weights [C_in][C_out][4][4][4]); a brute-force test pins its meaning.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

from .field import F64

SLOPE = 0.2


def weight_volume(layers, z: torch.Tensor, log_prior: torch.Tensor | None = None) -> torch.Tensor:
    """W^c [25][32][32][32] (channel, z, y, x) from layers = [(W_fc [C0][256], b_fc [C0]),
    (W_1 [C0][C1][4][4][4], b_1 [C1]), ..., (W_5 [C4][25][4][4][4], b_5 [25])]."""
    W, b = layers[0]
    h = F.leaky_relu(W @ z + b, SLOPE).reshape(1, -1, 1, 1, 1)
    n = len(layers) - 1
    for k, (W, b) in enumerate(layers[1:]):
        h = F.conv_transpose3d(h, W, b, stride=2, padding=1)
        if k < n - 1:
            h = F.leaky_relu(h, SLOPE)
    logits = h[0]
    if log_prior is not None:
        logits = logits + log_prior
    return torch.softmax(logits, dim=0)


def as_tensors(layers, requires_grad: bool = False):
    return [(torch.as_tensor(W, dtype=F64).clone().requires_grad_(requires_grad),
             torch.as_tensor(b, dtype=F64).clone().requires_grad_(requires_grad)) for W, b in layers]
