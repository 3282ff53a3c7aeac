"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np

import oracle as O
import sc_inputs as I

TWO_PI = 2.0 * np.pi


def gpu_context(**cfg):
    import torch
    from paper_1911_02366_gb300 import sc
    return sc.Context(stream=torch.cuda.current_stream().cuda_stream, **cfg)


def case(n, N, cfl=50.0, eps=1e-3, seed=0, bdf=1, **cfg):
    """Seeded TGV case set up on both sides: (Q, dt, oracle params, GPU context)."""
    Q, dt = I.tgv_state(n, N, cfl=cfl, eps=eps, seed=seed)
    p = O.Params(n=n, N=N, dt=dt, bdf=bdf)
    ctx = gpu_context(**cfg)
    ctx.sc_set_mesh(n, TWO_PI, N)
    ctx.sc_set_timestep(dt, bdf)
    return Q, dt, p, ctx


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def bf16_bits(x):
    """IEEE bfloat16 bit patterns (round to nearest even) of a float array, as uint16."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_values(bits):
    """float32 values of bfloat16 bit patterns."""
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)
