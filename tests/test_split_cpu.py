"""Halo-deepened domain split on the CPU: the slab geometry of the library
(an5d_split_geometry, host only) and its exchange schedule, run as two gloo
ranks that each advance their own slab with the CPU oracle and trade ghost
planes once per pass.  The gathered result must be the single-grid oracle
result bit for bit (the overlapped tiling of Section 2.3 applied to slabs)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2001_01473_gb300 import an5d, inputs


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(an5d.LIB_PATH):
        from paper_2001_01473_gb300 import build
        build.build()
    an5d.load()


@pytest.mark.parametrize("ndim,dims,R,bt,nsub", [(2, (100, 70), 1, 3, 4), (2, (37, 9), 2, 2, 3),
                                                 (3, (40, 6, 5), 1, 4, 3), (3, (12, 4, 4), 1, 1, 6),
                                                 (2, (9, 9), 1, 2, 2)])
def test_split_geometry_partitions_the_slow_axis(ndim, dims, R, bt, nsub):
    s = dims[0]
    g = [an5d.an5d_split_geometry(ndim, dims, R, bt, nsub, k) for k in range(nsub)]
    assert g[0]["a"] == 0 and g[-1]["b"] == s
    sizes = [x["b"] - x["a"] for x in g]
    assert max(sizes) - min(sizes) <= 1 and sorted(sizes, reverse=True) == sizes
    for k, x in enumerate(g):
        if k:
            assert x["a"] == g[k - 1]["b"]
        assert x["lo"] == max(0, x["a"] - bt * R)
        assert x["hi"] == min(s + 2 * R, x["b"] + bt * R + 2 * R)
        assert x["b"] - x["a"] >= bt * R + R


def test_split_geometry_rejects_thin_slabs_and_bad_arguments():
    with pytest.raises(an5d.An5dError) as e:
        an5d.an5d_split_geometry(2, (10, 10), 1, 4, 3, 0)     # 3 planes < bT R + R = 5
    assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
    for args in ((4, (10, 10), 1, 1, 2, 0), (2, (10, 10), 1, 1, 2, 2), (2, (10, 10), 0, 1, 2, 0),
                 (2, (10, 10), 1, 0, 2, 0), (2, (10, 10), 1, 1, 0, 0)):
        with pytest.raises(an5d.An5dError) as e:
            an5d.an5d_split_geometry(*args)
        assert e.value.status == an5d.AN5D_ERR_INVALID_ARG


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab_worker(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ndim, shape, R, bt, dims, T = case
        an5d.load()
        c32 = inputs.normalised_coeffs(inputs.coeff_count(ndim, shape, R), 0).astype(np.float32)
        u0 = inputs.field(dims, R, 1, "f32")
        geo = [an5d.an5d_split_geometry(ndim, dims, R, bt, world, k) for k in range(world)]
        me = geo[rank]
        loc = np.ascontiguousarray(u0[me["lo"]:me["hi"]])
        ldims = (me["hi"] - me["lo"] - 2 * R,) + tuple(dims[1:])
        passes = [bt] * (T // bt) + ([T % bt] if T % bt else [])
        for d in passes:
            loc = oracle.run_f32(ndim, shape, R, c32, ldims, loc, d)
            # one exchange per pass: the planes each neighbour holds but I own
            # go out, the planes I hold but a neighbour owns come in
            reqs, inbox = [], []
            for k in range(world):
                if k == rank:
                    continue
                o = geo[k]
                send0, send1 = max(o["lo"], me["a"] + R), min(o["hi"], me["b"] + R)
                recv0, recv1 = max(me["lo"], o["a"] + R), min(me["hi"], o["b"] + R)
                if send1 > send0:
                    reqs.append(dist.isend(torch.from_numpy(
                        np.ascontiguousarray(loc[send0 - me["lo"]:send1 - me["lo"]])), k))
                if recv1 > recv0:
                    buf = torch.empty((recv1 - recv0,) + loc.shape[1:], dtype=torch.float32)
                    reqs.append(dist.irecv(buf, k))
                    inbox.append((recv0, recv1, buf))
            for r in reqs:
                r.wait()
            for r0, r1, buf in inbox:
                loc[r0 - me["lo"]:r1 - me["lo"]] = buf.numpy()
        owned = torch.from_numpy(np.ascontiguousarray(loc[me["a"] + R - me["lo"]:me["b"] + R - me["lo"]]))
        if rank == 0:
            parts = [owned.numpy()]
            for k in range(1, world):
                buf = torch.empty((geo[k]["b"] - geo[k]["a"],) + loc.shape[1:], dtype=torch.float32)
                dist.recv(buf, k)
                parts.append(buf.numpy())
            out = u0.copy()
            out[R:dims[0] + R] = np.concatenate(parts)
            ref = oracle.run_f32(ndim, shape, R, c32, dims, u0, T)
            q.put(bool(np.array_equal(out.view(np.uint32), ref.view(np.uint32))))
        else:
            dist.send(owned, 0)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [(2, inputs.STAR, 1, 3, (40, 33), 8),
                                  (2, inputs.BOX, 2, 2, (30, 21), 5),
                                  (3, inputs.STAR, 1, 2, (16, 9, 11), 5)])
def test_two_rank_split_matches_single_grid(case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_slab_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(180)
        assert p.exitcode == 0
    assert q.get(timeout=10) is True
