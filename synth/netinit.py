"""Seeded initial parameters of the warm-start network (an input: the library draws no random numbers).

He-uniform weights, bound sqrt(6 / fan_in) with fan_in = C_in * 27, zero biases, for 3x3x3 convolution
layers with the given channel counts, packed per layer as W[co][ci][tz][ty][tx] then bias[co] (float32).
"""
import numpy as np

CHANNELS = (5, 32, 32, 32, 3)


def init_params(seed, channels=CHANNELS):
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in zip(channels[:-1], channels[1:]):
        bound = np.sqrt(6.0 / (ci * 27))
        parts.append(rng.uniform(-bound, bound, size=co * ci * 27))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)
