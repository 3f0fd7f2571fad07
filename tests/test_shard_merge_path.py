"""Row sharding of SpMV over ranks by the merge path (the multi-GPU design, tested on
CPU with gloo, world sizes 2 and 3): rank r owns the r-th equal share of rows + atoms,
split on its diagonals by the oracle's merge-path search; it sums the atoms of its
share into the rows they belong to, the boundary rows' partial sums meet in one
all-reduce, and the result equals the full SpMV exactly (integer-valued inputs make
every FP64 sum exact).  The same holds when the shares are cut with row ends weighted
(the row_weight cut: equal cost w * rows + atoms per rank)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import workloads as W
    m = W.powerlaw(3000, 2500, 60_000, lmax=2000, plant_long=False, seed=17)
    rng = np.random.default_rng(3)
    v = rng.integers(-8, 9, m.nnz).astype(np.float32)
    x = rng.integers(-8, 9, m.num_cols).astype(np.float32)
    return m, v, x


def _worker(rank, world, port, out, w=1):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, v, x = _case()
    R, N = m.num_rows, m.nnz
    items = R + N
    if w == 1:
        d0, d1 = rank * items // world, (rank + 1) * items // world
    else:
        # start and end diagonal of each rank's weighted share (one tile spanning the whole share)
        diag = oracle.weighted_diagonals(m.rp, w, world, w * R + N + 1, 1).reshape(world, 2)
        d0, d1 = int(diag[rank, 0]), int(diag[rank, 1])
    (i0, j0), (i1, j1) = oracle.merge_split(d0, m.rp), oracle.merge_split(d1, m.rp)
    # this rank's atoms [j0, j1) summed into their rows (the boundary rows partly)
    y = np.zeros(R, dtype=np.float64)
    row_of = oracle.row_of_atom(m.rp)
    for k in range(j0, j1):
        y[row_of[k]] += float(v[k]) * float(x[m.ci[k]])
    yt = torch.from_numpy(y)
    dist.all_reduce(yt)  # boundary rows: the partial sums of adjacent ranks meet here
    y_ref, _ = oracle.spmv(m.rp, m.ci, v, x)
    out[rank] = (bool(np.array_equal(yt.numpy(), y_ref)), int(i0), int(j0), int(i1), int(j1))
    dist.destroy_process_group()


def _run(world, w=1):
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out, w)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        return [out[r] for r in range(world)]


def test_merge_path_shards_sum_to_the_full_spmv():
    for world, w in ((2, 1), (3, 1), (3, 4)):
        res = _run(world, w)
        assert all(ok for ok, *_ in res)
        # the shards tile the merge path: each starts where the previous ended
        for (_, _, _, i1, j1), (_, i0, j0, _, _) in zip(res, res[1:]):
            assert (i1, j1) == (i0, j0)
        m, _, _ = _case()
        assert res[0][1:3] == (0, 0) and res[-1][3:] == (m.num_rows, m.nnz)
