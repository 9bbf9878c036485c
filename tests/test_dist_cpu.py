"""The multi-GPU path of the benchmark on CPU: two processes over gloo (world
size 2). The work shards into independent maps, so the only collectives are
the max-over-ranks of the step time and the agreement on the reported path;
each rank draws its own maps and solves them alone (checked here with the FP64
oracle on small maps)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    import synth
    from oracle import physics as ph
    from oracle import solve as so
    dev = torch.device("cpu")
    assert bench._dist() == (ws, rank, rank)
    # each rank's shard: its own maps
    w, pd, pl, s = synth.batch_inputs(32, 2, device="cpu", seed=bench.rank_seed(rank))
    # slowest rank decides the job's time; rank 0's choice is reported by all
    t_local = 1.0 + rank
    t_max = bench._max_over_ranks(t_local, ws, dev)
    names = ["a", "b", "c"]
    chosen = bench.agree_on(names, names[rank + 1], ws, dev)
    # solve the shard locally (no data exchange)
    st, phy = w.stack, w.physics
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    th, _, it = so.picard(lambda x: so.spectral_convolve(Kt, x), pd[0].double().numpy(),
                          pl[0].double().numpy(), s[0].double().numpy(), phy.beta_per_K,
                          phy.alpha_per_K, tol=1e-8)
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), pd=pd.numpy(), t_max=t_max,
             chosen=names.index(chosen), theta=th, rate=bench.whole_job_rate(ws, 2, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_maps_and_agree_on_time_and_path(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    # disjoint shards: the ranks drew different maps
    assert not np.array_equal(r0["pd"], r1["pd"])
    # the job's time is the slowest rank's, on every rank
    assert float(r0["t_max"]) == float(r1["t_max"]) == 2.0
    # every rank reports rank 0's path
    assert int(r0["chosen"]) == int(r1["chosen"]) == 1
    # whole-job rate = all ranks' maps over the slowest time
    assert float(r0["rate"]) == pytest.approx(2 * 2 / 2.0)
    # each rank's result is its own map's solution (finite, positive rise)
    for r in (r0, r1):
        assert np.all(np.isfinite(r["theta"])) and r["theta"].min() > 0


def test_rank_seed_is_deterministic_and_distinct():
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    import bench
    assert bench.rank_seed(0) != bench.rank_seed(1)
    assert bench.rank_seed(3) == bench.rank_seed(3)
    assert bench.whole_job_rate(1, 4096, 0.01) == pytest.approx(409600.0)
