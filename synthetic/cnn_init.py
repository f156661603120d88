"""Seeded initial weights of the learned-augmentation network (the U-Net).

Random numbers the method draws are inputs: both the CUDA library (through
rcg_learn_set_weights) and the oracle start from this vector.  Layout: for
each layer (Cin, Cout) in order, W [Cout][Cin][27] then b [Cout]; normal
weights with variance 2 / (27 Cin) (He scaling for ReLU layers), zero biases.
"""
import numpy as np

# (input channels, output channels) of the ten 3x3x3 convolutions, in order
LAYERS = ((2, 16), (16, 16), (16, 32), (32, 32), (32, 64), (96, 32), (32, 32), (48, 16), (16, 16), (16, 1))


def init_weights(seed=0, layers=LAYERS):
    rng = np.random.default_rng(10_000 + seed)
    parts = []
    for ci, co in layers:
        parts.append(rng.standard_normal(co * ci * 27) * np.sqrt(2.0 / (27 * ci)))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)
