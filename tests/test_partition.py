"""The slab partitioning of the path across ranks, checked on CPU ranks (gloo,
world size 2) with the FP64 oracle's own stage primitives.

The z transform (F_u1D) works on x-slabs of the volume, the plane transform
(F_u2D) on kv-slabs of the spectrum, so L_hat needs one all-to-all exchange
of u1 (x-slab -> kv-slab) and L_hat^H the reverse one; the TV gradient on
x-slabs needs a one-plane halo; the CG / ADMM scalars are FP64 sums reduced
across ranks.  Every partitioned result is compared with the single-process
oracle.  The all-to-all is written as pairwise send / receive.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import lamino as olam
from oracle import tv as otv
from oracle import usfft

N, NZ, H, W, T = 16, 8, 8, 16, 6


def _geom():
    theta = np.linspace(0, 2 * np.pi, T, endpoint=False) + 0.1
    return olam.Geometry(n1=N, n0=NZ, n2=N, h=H, w=W, theta=theta, phi=0.5)


def _inputs():
    rng = np.random.default_rng(5)
    u = rng.standard_normal((N, NZ, N))
    r = rng.standard_normal((T, H, W)) + 1j * rng.standard_normal((T, H, W))
    return u, r


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _all_to_all(blocks, rank, world):
    """blocks[j] goes to rank j; returns the blocks received, by source rank."""
    out = [None] * world
    out[rank] = blocks[rank]
    for j in range(world):
        if j == rank:
            continue
        send = torch.from_numpy(np.ascontiguousarray(blocks[j]).view(np.float64).copy())
        recv = torch.empty_like(send)
        reqs = [dist.isend(send, j), dist.irecv(recv, j)]
        for q in reqs:
            q.wait()
        out[j] = recv.numpy().view(np.complex128).reshape(blocks[j].shape)
    return out


def _gather(x, world):
    parts = [torch.empty_like(x) for _ in range(world)]
    dist.all_gather(parts, x)
    return parts


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = _geom()
    u, r = _inputs()
    xs = [slice(j * N // world, (j + 1) * N // world) for j in range(world)]
    ks = [slice(j * H // world, (j + 1) * H // world) for j in range(world)]
    xi_x, xi_y, _ = olam.slice_frequencies(g)
    res = {}

    # ---- L_hat: F_u1D on my x-slab, all-to-all to kv-slabs, F_u2D per plane
    u1_x = olam.f_u1d(u[xs[rank]], g)                                  # [n/W, h, n]
    got = _all_to_all([u1_x[:, ks[j], :] for j in range(world)], rank, world)
    u1_k = np.concatenate(got, axis=0)                                 # [n, h/W, n]
    d_k = np.empty((T, u1_k.shape[1], W), dtype=np.complex128)
    for i, kv in enumerate(range(H)[ks[rank]]):
        P = usfft.usfft2d_grid(u1_k[:, i, :], g.m, g.R)
        d_k[:, i, :] = usfft.usfft2d_gather(P, xi_x[:, kv, :], xi_y[:, kv, :], g.m, g.R)
    res["lhat"] = np.abs(d_k - olam.lhat(u, g)[:, ks[rank], :]).max()

    # ---- L_hat^H: type-1 per plane on my kv-slab, all-to-all back, F*_u1D
    a_k = np.empty((N, H // world, N), dtype=np.complex128)
    for i, kv in enumerate(range(H)[ks[rank]]):
        a_k[:, i, :] = usfft.usfft2d_type1(r[:, kv, :], xi_x[:, kv, :], xi_y[:, kv, :], N, N, g.m, g.R)
    got = _all_to_all([a_k[xs[j]] for j in range(world)], rank, world)
    a_x = np.concatenate(got, axis=1)                                  # [n/W, h, n]
    adj_x = olam.f_u1d_adj(a_x, g).real
    res["lhat_adj"] = np.abs(adj_x - olam.lhat_adj(r, g)[xs[rank]]).max()

    # ---- TV gradient on x-slabs with a one-plane halo from the next rank
    my = u[xs[rank]]
    halo = torch.zeros((NZ, N), dtype=torch.float64)
    if rank > 0:
        dist.send(torch.from_numpy(np.ascontiguousarray(my[0])), rank - 1)
    if rank < world - 1:
        dist.recv(halo, rank + 1)
    ext = np.concatenate([my, halo.numpy()[None]], axis=0) if rank < world - 1 else my
    gx = np.zeros_like(my)
    gx[: ext.shape[0] - 1] = ext[1:] - ext[:-1]
    if rank == world - 1:
        gx[-1] = 0.0                                                   # Neumann end
    res["grad_x"] = np.abs(gx - otv.grad(u)[0][xs[rank]]).max()

    # ---- an FP64 CG scalar, ||L_hat u||^2, as partial sums reduced across ranks
    part = torch.tensor([np.vdot(d_k, d_k).real], dtype=torch.float64)
    dist.all_reduce(part)
    full = np.vdot(olam.lhat(u, g), olam.lhat(u, g)).real
    res["norm"] = abs(part.item() - full) / full
    out[rank] = res
    dist.destroy_process_group()


def test_slab_partitioned_path_matches_single_process_oracle():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        res = out[rank]
        assert res["lhat"] < 1e-12
        assert res["lhat_adj"] < 1e-12
        assert res["grad_x"] == 0.0
        assert res["norm"] < 1e-14


def test_slab_bounds_cover_every_index_once():
    for world in (2, 4):
        xs = [range(N)[j * N // world:(j + 1) * N // world] for j in range(world)]
        ks = [range(H)[j * H // world:(j + 1) * H // world] for j in range(world)]
        assert sorted(i for s in xs for i in s) == list(range(N))
        assert sorted(i for s in ks for i in s) == list(range(H))


if __name__ == "__main__":
    pytest.main([__file__, "-q"])
