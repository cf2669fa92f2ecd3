"""Shared set-up for the GPU parity tests: seeded inputs written into a Box
(the C-ABI binding) and the same bytes handed to the oracle."""
import numpy as np

import oracle as O
from paper_2312_11448_gb300.inputs import density_field, doppler_quantiles, velocity_field


def make_fields(n, sigma=0.8, sigma_v=1.0, seed=1):
    d = density_field(n, sigma, seed).ravel()
    U = velocity_field(n, sigma_v, seed) if sigma_v > 0 else np.zeros((n ** 3, 3))
    return d, U


def new_box(n, precision, mixing="tally", n_packets=100_000, sigma=0.8, sigma_v=1.0, seed=1, rng_seed=7, n_sub=1):
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(n, sigma, sigma_v, seed)
    box = rec.Box(n, d, U, n_packets, precision=precision, mixing=mixing, seed=rng_seed, n_sub=n_sub)
    return box


def field_dtype(box):
    return np.float32 if box.precision == "mixed" else np.float64


def set_state(box, x, T, tally=None, emis=None):
    """Write a state into the box's device buffers (exact bytes)."""
    import torch
    fdt = field_dtype(box)
    box.stream.synchronize()
    box.x.copy_(torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)))
    box.T.copy_(torch.as_tensor(np.ascontiguousarray(T, dtype=fdt)))
    if tally is not None:
        box.tally.copy_(torch.as_tensor(np.ascontiguousarray(tally, dtype=np.uint32).view(np.int32)))
    if emis is not None:
        box.emis.copy_(torch.as_tensor(np.ascontiguousarray(emis, dtype=fdt)))
    torch.cuda.synchronize()


def oracle_fields(box):
    """(delta, U [n3,3], vel4) exactly as stored on the device, widened to float64."""
    d = box.host("delta").astype(np.float64)
    v4 = box.host("vel4")
    return d, v4[:, :3].astype(np.float64), v4


def quantiles(box):
    q = doppler_quantiles()
    return q.astype(field_dtype(box))
