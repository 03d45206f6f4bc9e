"""FP64 CPU oracle of the learned initial guess network (test infrastructure).

Only tests/ (and bench.py's CPU legs) may import this module.  It is the
plain reference the CUDA network is checked against and shares no code with
it.  The network (the paper has no learned part; see include/qumond_guess.h
for the specification both sides follow): a 3-D U-Net on S^3 voxels with
16 input channels, levels S, S/2, S/4, S/8 with 16, 32, 64, 128 channels,
every convolution 3x3x3 with zero padding + bias + ReLU, two per level down
(2x2x2 average pooling between levels) and two per level up
(nearest-neighbour upsampling, then the concatenation [upsampled, skip]),
and a 1x1x1 head 16 -> 1 without ReLU.

Written with plain PyTorch CPU operations in float64: the convolution is
torch's cross-correlation (a library primitive), pooling and upsampling are
reshapes and means, and the gradient is torch.autograd of the loss.  The
weights are BF16 by definition of the network, so the oracle rounds them to
BF16 (round to nearest even) before use, as the GPU does; activations stay
FP64 here, so the comparison measures the GPU's BF16 activation rounding.

Layouts: a parameter vector holds, per layer, W[cout][27][cin] with tap
t = (dz+1)*9 + (dy+1)*3 + (dx+1) reading input voxel (x+dx, y+dy, z+dz),
then b[cout]; then the head's w[16] and b.  A voxel array of an S^3 level
is indexed [z][y][x].
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

# (cin, cout) of the 14 convolutions: encoder levels 0-3, then decoder levels 2, 1, 0
LAYERS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
          (192, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]


def num_params() -> int:
    return sum(27 * ci * co + co for ci, co in LAYERS) + 17


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_weight(W, cin, cout):
    """W[co][tap][ci] (flat), tap = kz*9 + ky*3 + kx  ->  torch weight[co][ci][kz][ky][kx]."""
    w = np.asarray(W, dtype=np.float64).reshape(cout, 3, 3, 3, cin)
    return torch.from_numpy(w.transpose(0, 4, 1, 2, 3).copy())


def unpack(params, round_weights=True):
    """Split a parameter vector into [(conv weight, b)] per layer and the head (w, b).
    round_weights: the convolution weights are the BF16 values of the FP32 parameters."""
    p = np.asarray(params, dtype=np.float64)
    assert p.size == num_params()
    out = []
    o = 0
    for ci, co in LAYERS:
        w = p[o:o + 27 * ci * co]
        if round_weights:
            w = bf16_round(w.astype(np.float32))
        o += 27 * ci * co
        b = p[o:o + co].copy()
        o += co
        out.append((conv_weight(w, ci, co), torch.from_numpy(b)))
    head_w = torch.from_numpy(p[o:o + 16].copy())
    head_b = torch.tensor(float(p[o + 16]), dtype=torch.float64)
    return out, (head_w, head_b)


def conv3(x, w, b):
    """x: [cin][S][S][S] -> [cout][S][S][S]; out[co, z, y, x] = b + sum w[co, ci, kz, ky, kx] x[ci, z+kz-1, ...]."""
    return F.conv3d(x[None], w, b, padding=1)[0]


def pool(x):
    c, s = x.shape[0], x.shape[1]
    return x.reshape(c, s // 2, 2, s // 2, 2, s // 2, 2).mean(dim=(2, 4, 6))


def up(x):
    return x.repeat_interleave(2, dim=1).repeat_interleave(2, dim=2).repeat_interleave(2, dim=3)


def network_input(sample, flag):
    """The 16-channel input of a sample: its rho and Phi_N channels (any float array
    of 3 S^3 values in voxel order), the box flag, zeros."""
    s3 = sample.size // 3
    S = round(s3 ** (1.0 / 3.0))
    x = torch.zeros((16, S, S, S), dtype=torch.float64)
    x[0] = torch.from_numpy(np.asarray(sample[:s3], dtype=np.float64).reshape(S, S, S))
    x[1] = torch.from_numpy(np.asarray(sample[s3:2 * s3], dtype=np.float64).reshape(S, S, S))
    x[2] = float(flag)
    return x


def bf16_acts(t):
    """An activation stored in BF16 (round to nearest even), kept as float64."""
    return t.to(torch.bfloat16).to(torch.float64)


def forward(layers, head, x, store=None, terms=False):
    """Network output y [S][S][S] for input x [16][S][S][S].

    store: None keeps every activation in float64; bf16_acts stores each one in
    BF16 at the points where the network's definition holds activations in
    BF16 (every convolution's output after ReLU, every pooled level; the
    upsampled copies and the concatenations are those values unchanged).
    terms: also return T[z][y][x] = sum over the head's channels c of
    |w_c d0_c|, the magnitude of the output's terms."""
    keep = store if store is not None else (lambda t: t)

    def c(i, t):
        return keep(torch.relu(conv3(t, *layers[i])))

    def p(t):
        return keep(pool(t))
    e0 = c(1, c(0, x))
    e1 = c(3, c(2, p(e0)))
    e2 = c(5, c(4, p(e1)))
    b3 = c(7, c(6, p(e2)))
    d2 = c(9, c(8, torch.cat([up(b3), e2])))
    d1 = c(11, c(10, torch.cat([up(d2), e1])))
    d0 = c(13, c(12, torch.cat([up(d1), e0])))
    hw, hb = head
    y = torch.einsum("c,czyx->zyx", hw, d0) + hb
    if terms:
        return y, torch.einsum("c,czyx->zyx", hw.abs(), d0.abs())
    return y


def predict(params, sample, flag, round_weights=True, store=None, terms=False):
    """Output voxels (flat, x fastest); with terms=True also the per-voxel term magnitudes."""
    layers, head = unpack(params, round_weights)
    with torch.no_grad():
        out = forward(layers, head, network_input(sample, flag), store=store, terms=terms)
    if terms:
        return out[0].numpy().ravel(), out[1].numpy().ravel()
    return out.numpy().ravel()


def loss_and_gradients(params, samples, flags, round_weights=True):
    """Batch loss (mean over samples of the mean squared error against each
    sample's third channel) and its gradient in the parameter layout (with
    respect to the weights as used, i.e. the BF16 values when rounded)."""
    layers, head = unpack(params, round_weights)
    leaves = []
    for w, b in layers:
        w.requires_grad_(True)
        b.requires_grad_(True)
        leaves += [w, b]
    head[0].requires_grad_(True)
    head[1].requires_grad_(True)
    total = torch.zeros((), dtype=torch.float64)
    for smp, fl in zip(samples, flags):
        smp = np.asarray(smp, dtype=np.float64)
        s3 = smp.size // 3
        y = forward(layers, head, network_input(smp, fl)).reshape(-1)
        t = torch.from_numpy(smp[2 * s3:])
        total = total + torch.mean((y - t) ** 2)
    total = total / len(samples)
    total.backward()
    g = []
    for (w, b), (ci, co) in zip(layers, LAYERS):
        # weight[co][ci][kz][ky][kx] -> W[co][tap][ci]
        g.append(w.grad.numpy().transpose(0, 2, 3, 4, 1).reshape(-1))
        g.append(b.grad.numpy())
    g.append(head[0].grad.numpy())
    g.append(np.array([head[1].grad.item()]))
    return float(total.item()), np.concatenate(g)


def layer_slices():
    """(name, slice) of every weight and bias block of the parameter vector, and the head."""
    out = []
    o = 0
    for i, (ci, co) in enumerate(LAYERS):
        out.append(("W%d" % i, slice(o, o + 27 * ci * co)))
        o += 27 * ci * co
        out.append(("b%d" % i, slice(o, o + co)))
        o += co
    out.append(("head", slice(o, o + 17)))
    return out
