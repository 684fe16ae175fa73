"""Host logic of bench.py (CPU only): kernel byte/flop models, replica
aggregation across ranks (gloo, world size 2), JSON plumbing helpers."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_kernel_models_scale_with_rhs_and_precision():
    m1 = bench.kernel_models(1000, [10, 11, 12], [20, 24, 24], 80000, 27000, 27, 1, 16)
    m4 = bench.kernel_models(1000, [10, 11, 12], [20, 24, 24], 80000, 27000, 27, 4, 16)
    m1s = bench.kernel_models(1000, [10, 11, 12], [20, 24, 24], 80000, 27000, 27, 1, 8)
    for k in ("fft_z_fwd", "fft_y_fwd", "fft_x_conv", "fft_y_inv", "fft_z_inv"):
        assert m4[k][1] == pytest.approx(4 * m1[k][1])  # flops linear in the batch
        assert m1s[k][0] < m1[k][0]  # complex64 moves fewer bytes
    # x pass: two transforms of length Lx per (ky, kz) row and grid, plus the product
    nx, Lx, Ly, Lz = 10, 20, 24, 24
    assert m1["fft_x_conv"][1] == pytest.approx(4 * Ly * Lz * (10 * Lx * np.log2(Lx) + 6 * Lx))


def test_projection_model_counts_the_projected_nodes():
    """With a group list the projection writes only the nodes of its groups;
    the interpolation reads only the touched nodes; both default to the grid."""
    n, L = [10, 11, 12], [20, 24, 24]
    Nc = 10 * 11 * 12
    full = bench.kernel_models(1000, n, L, 80000, 27000, 27, 2, 8)
    part = bench.kernel_models(1000, n, L, 80000, 27000, 27, 2, 8, touched=400, projected=320)
    G, e = 8, 8
    assert full["proj_gather"][0] - part["proj_gather"][0] == (Nc - 320) * (4 + G * e)
    assert full["interp_near"][0] - part["interp_near"][0] == G * (Nc - 400) * e
    assert part["proj_gather"][1] == full["proj_gather"][1]  # same arithmetic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r pretends its timed products took (100 + 50 r) ms
    total, value = bench.aggregate(100.0 + 50.0 * rank, steps=10, nrhs=2, world=world, device="cpu")
    q.put((rank, total, value))
    dist.destroy_process_group()


def test_replica_aggregation_takes_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in out:
        assert total == pytest.approx(150.0)  # max over ranks
        assert value == pytest.approx(world * 10 * 2 / 0.150)


def test_single_rank_aggregation_is_local():
    total, value = bench.aggregate(200.0, steps=20, nrhs=1, world=1)
    assert total == 200.0 and value == pytest.approx(100.0)


def test_oracle_sample_pieces_make_up_products():
    """The oracle's bounded timing sample: pieces cycle through the four grid
    components, and four pieces count as one product."""
    from aim_inputs import plate_mesh, random_complex

    v, t = plate_mesh(1.0, 9)
    o = bench.OracleSample(v, t, sample_rows=16)
    x = random_complex((1, o.N), 3)
    comps = []
    for _ in range(5):
        comps.append(o.comp)
        o.piece(x)
    assert comps == [0, 1, 2, 3, 0]
    r = o.result(warm=1)
    assert r["value"] == pytest.approx(0.25 * 4 / sum(o.t[1:]))
    assert r["kind"] == "oracle" and r["cores"] == os.cpu_count() and r["unit"] == "matvec/s"
