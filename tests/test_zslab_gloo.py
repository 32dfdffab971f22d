"""Exchange step of the decomposition of one operator over ranks: Krylov vectors by lateral
columns, the lateral contrast stage by absorber planes.  Checked with gloo ranks on CPU (world
sizes 2 and 3, uneven splits): every rank receives exactly the planes it owns from every other
rank's columns, the inverse exchange restores the column distribution, the distributed dot
product is the global one, and the lateral contrast stage (Sec. 2.2: IFFT2, times the plane's
permittivity contrast, FFT2) run plane by plane on the plane distribution and brought back gives
the undistributed result on every rank's columns."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, lead, planes, columns, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2607_25330_b300.zslab import ColumnPlaneExchange, distributed_dot
        g = torch.Generator().manual_seed(5)
        full = torch.complex(torch.randn(lead, planes, columns, generator=g, dtype=torch.float64),
                             torch.randn(lead, planes, columns, generator=g, dtype=torch.float64))
        ex = ColumnPlaneExchange(planes, columns, world, rank)
        c0, c1 = ex.my_columns()
        z0, z1 = ex.my_planes()
        x_cols = full[:, :, c0:c1].contiguous()
        x_pl = ex.to_planes(x_cols)
        ok_planes = torch.equal(x_pl, full[:, z0:z1, :])
        back = ex.to_columns(x_pl)
        ok_back = torch.equal(back, x_cols)
        local = float((x_cols.abs() ** 2).sum())
        tot = float(distributed_dot([local])[0])
        q.put((rank, ok_planes, ok_back, tot, float((full.abs() ** 2).sum())))
    finally:
        dist.destroy_process_group()


def _contrast(g, deps, ny, nx):
    """k0^2-free contrast stage on lateral spectra g [lead][planes][ny*nx] with deps [planes][ny][nx]."""
    lead, planes = g.shape[0], g.shape[1]
    f = torch.fft.ifft2(g.reshape(lead, planes, ny, nx), norm="ortho")
    return torch.fft.fft2(f * deps, norm="ortho").reshape(lead, planes, ny * nx)


def _rank_contrast(rank, world, port, lead, planes, ny, nx, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2607_25330_b300.zslab import ColumnPlaneExchange
        g = torch.Generator().manual_seed(9)
        full = torch.complex(torch.randn(lead, planes, ny * nx, generator=g, dtype=torch.float64),
                             torch.randn(lead, planes, ny * nx, generator=g, dtype=torch.float64))
        deps = torch.complex(torch.rand(planes, ny, nx, generator=g, dtype=torch.float64),
                             0.1 * torch.rand(planes, ny, nx, generator=g, dtype=torch.float64))
        ex = ColumnPlaneExchange(planes, ny * nx, world, rank)
        c0, c1 = ex.my_columns()
        z0, z1 = ex.my_planes()
        y_pl = _contrast(ex.to_planes(full[:, :, c0:c1].contiguous()), deps[z0:z1], ny, nx)
        y_cols = ex.to_columns(y_pl)
        ref = _contrast(full, deps, ny, nx)[:, :, c0:c1]
        q.put((rank, float((y_cols - ref).abs().max()), float(ref.abs().max())))
    finally:
        dist.destroy_process_group()


def _run(world, lead, planes, columns, target=None, args=None):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    target = target or _rank
    args = args or (lead, planes, columns)
    procs = [ctx.Process(target=target, args=(r, world, port) + tuple(args) + (q,)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    return sorted(q.get(timeout=10) for _ in range(world))


def test_column_plane_exchange_two_ranks():
    for rank, ok_planes, ok_back, tot, ref in _run(2, 6, 31, 40):
        assert ok_planes and ok_back, rank
        assert abs(tot - ref) <= 1e-12 * ref


def test_column_plane_exchange_three_ranks_uneven():
    for rank, ok_planes, ok_back, tot, ref in _run(3, 3, 7, 17):
        assert ok_planes and ok_back, rank
        assert abs(tot - ref) <= 1e-12 * ref


def test_even_split_covers_the_range():
    from paper_2607_25330_b300.zslab import even_split
    for n, p in ((31, 2), (7, 3), (5, 5), (4, 3)):
        parts = even_split(n, p)
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        assert max(e - s for s, e in parts) - min(e - s for s, e in parts) <= 1


def test_contrast_stage_on_the_plane_distribution():
    # 3 components x 5 absorber planes of a 12 x 10 lateral grid over 3 ranks (uneven splits)
    out = _run(3, 0, 0, 0, target=_rank_contrast, args=(3, 5, 12, 10))
    for rank, err, ref in out:
        assert err <= 1e-13 * ref, (rank, err, ref)
