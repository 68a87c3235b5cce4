"""Host logic of the horizontal domain decomposition (no GPU): the partition plan built by
the library from host connectivity, checked against an independent breadth-first search,
and a halo exchange between two gloo ranks (world size 2) driven by the plan."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _tables(bis):
    import oracle as O
    g = O.build_grid(2, bis)
    return g, (g.c2e, g.e2c, g.c2v, g.v2c, g.vdeg)


def _rings(g, start, rings):
    """Cells within `rings` vertex rings of the set `start` (a ring adds the cells that share
    a vertex with the set), by plain breadth-first search."""
    cells_of_vertex = [set() for _ in range(g.nv)]
    for c in range(g.nc):
        for v in g.c2v[c]:
            cells_of_vertex[v].add(c)
    seen = set(start)
    front = set(start)
    for _ in range(rings):
        nxt = set()
        for c in front:
            for v in g.c2v[c]:
                nxt |= cells_of_vertex[v]
        nxt -= seen
        seen |= nxt
        front = nxt
    return seen


@pytest.mark.parametrize("nparts,rings", [(3, 3), (4, 2)])
def test_partition_plan_against_breadth_first_search(built_lib, nparts, rings):
    from paper_2511_02021_gb300 import capi as C
    g, tabs = _tables(2)
    owned_by = [np.full(n, -1) for n in (g.nc, g.ne, g.nv)]
    plans = [C.icon_partition_plan(*tabs, nparts, p, rings) for p in range(nparts)]
    for p, (counts, loc, own, oix) in enumerate(plans):
        nl = counts[3:]
        parts = np.split(loc, [nl[0], nl[0] + nl[1]])
        owners = np.split(own, [nl[0], nl[0] + nl[1]])
        # owned cells: the contiguous Morton range of the part
        lo, hi = p * g.nc // nparts, (p + 1) * g.nc // nparts
        assert np.array_equal(parts[0][:counts[0]], np.arange(lo, hi))
        # local cells: exactly the cells within `rings` vertex rings of the owned ones
        assert set(parts[0].tolist()) == _rings(g, range(lo, hi), rings)
        # local edges and vertices: those of the local cells
        assert set(parts[1].tolist()) == set(g.c2e[parts[0]].ravel().tolist())
        assert set(parts[2].tolist()) == set(g.c2v[parts[0]].ravel().tolist())
        for t in range(3):
            own_t, halo_t = parts[t][:counts[t]], parts[t][counts[t]:]
            assert np.all(np.diff(own_t) > 0) and np.all(np.diff(halo_t) > 0)
            assert np.all(owners[t][:counts[t]] == p) and np.all(owners[t][counts[t]:] != p)
            assert np.all(owned_by[t][own_t] == -1)
            owned_by[t][own_t] = p
    # every entity has exactly one owner: edges by their first (lower) cell, vertices by
    # their lowest incident cell
    assert all(np.all(o >= 0) for o in owned_by)
    cell_owner = owned_by[0]
    assert np.array_equal(owned_by[1], cell_owner[g.e2c[:, 0]])
    vmin = np.array([g.v2c[v, :g.vdeg[v]].min() for v in range(g.nv)])
    assert np.array_equal(owned_by[2], cell_owner[vmin])
    # the owner index of a halo entity is its position in the owner's local order
    for p, (counts, loc, own, oix) in enumerate(plans):
        for i in range(len(loc)):
            q = own[i]
            t = 0 if i < counts[3] else (1 if i < counts[3] + counts[4] else 2)
            base_q = [0, plans[q][0][3], plans[q][0][3] + plans[q][0][4]][t]
            assert plans[q][1][base_q + oix[i]] == loc[i]


def test_partition_plan_rejects_bad_arguments(built_lib):
    from paper_2511_02021_gb300 import capi as C
    _, tabs = _tables(0)
    for nparts, part, rings in [(0, 0, 3), (2, 2, 3), (2, -1, 3), (2, 0, 17)]:
        with pytest.raises(C.IconError) as ei:
            C.icon_partition_plan(*tabs, nparts, part, rings)
        assert ei.value.status == C.ICON_EINVAL


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as td
    from paper_2511_02021_gb300 import capi as C
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, tabs = _tables(2)
        counts, loc, own, oix = C.icon_partition_plan(*tabs, world, rank, 3)
        nlc = int(counts[3])
        cells, owner, oidx = loc[:nlc], own[:nlc], oix[:nlc]
        # a field known only on the owned rows; halo rows start as NaN
        f = np.full(nlc, np.nan)
        f[:counts[0]] = 1.5 * cells[:counts[0]] + 0.25
        other = 1 - rank
        need = np.nonzero(owner == other)[0]                     # halo rows owned by the other rank
        req = torch.from_numpy(oidx[need].astype(np.int64))
        n_mine = torch.tensor([len(need)], dtype=torch.int64)
        n_theirs = torch.zeros(1, dtype=torch.int64)
        # point-to-point, lower rank sends first: request sizes, requests, then the values
        if rank == 0:
            td.send(n_mine, other); td.recv(n_theirs, other)
        else:
            td.recv(n_theirs, other); td.send(n_mine, other)
        theirs = torch.zeros(int(n_theirs.item()), dtype=torch.int64)
        if rank == 0:
            td.send(req, other); td.recv(theirs, other)
        else:
            td.recv(theirs, other); td.send(req, other)
        reply = torch.from_numpy(f[theirs.numpy()].copy())        # rows I own that the other needs
        got = torch.zeros(len(need), dtype=torch.float64)
        if rank == 0:
            td.send(reply, other); td.recv(got, other)
        else:
            td.recv(got, other); td.send(reply, other)
        f[need] = got.numpy()
        q.put((rank, bool(np.all(np.isfinite(f))), bool(np.array_equal(f, 1.5 * cells + 0.25)), len(need)))
    finally:
        td.destroy_process_group()


def test_halo_exchange_between_two_gloo_ranks(built_lib):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, finite, exact, nhalo in res:
        assert finite and exact and nhalo > 0, (rank, finite, exact, nhalo)
