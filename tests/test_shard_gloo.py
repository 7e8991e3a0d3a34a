"""The N-process path on CPU: two gloo ranks shard independent task sets.

Each rank draws its own batch (seed offset by rank), decides it (here with
the CPU oracle, since there is no GPU), and the ranks exchange only scalars:
the max of their step times and the sum of their counts.  The test checks
that the ranks' batches are disjoint and reproducible, that the reductions
return the max / sum, and that the shards' contiguous bounds tile the range.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import oracle
    from paper_2105_10312_gb300 import gen_tasksets, shard
    from paper_2105_10312_gb300 import workloads as W

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = shard.dist_env()
    assert (r, w, local) == (rank, world, rank)
    p = W.gen_params("batch", nsets=400)
    p["seed"] = shard.rank_seed(p["seed"], r)
    s = gen_tasksets(**p)
    md = W.model("batch")
    res = oracle.allocate(s, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"])
    shard.barrier()
    t_mine = 1.0 + rank  # a stand-in step time per rank
    t_max = shard.max_over_ranks(t_mine)
    n_sum = shard.sum_over_ranks(int(res["verdict"].sum()))
    q.put((rank, t_max, n_sum, int(res["verdict"].sum()), int(s["T"][:16].sum()),
           [shard.shard_bounds(1003, k, world) for k in range(world)]))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_data_collectives():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(o[1] == 2.0 for o in out)                    # max of 1.0 and 2.0
    assert all(o[2] == out[0][3] + out[1][3] for o in out)  # sum of the ranks' counts
    assert out[0][4] != out[1][4]                            # disjoint batches
    bounds = out[0][5]
    assert bounds[0][0] == 0 and bounds[-1][1] == 1003
    assert all(bounds[k][1] == bounds[k + 1][0] for k in range(world - 1))
