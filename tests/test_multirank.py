"""The N > 1 bench path on CPU: two ranks over gloo.  The GPU path runs
independent replicas (no data-path collective); what crosses ranks is the
barrier around the timed region and the max over ranks of the step time."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    bench.barrier(world)
    m = bench.max_over_ranks(1.5 + rank, world)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"max": m}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert json.load(open(tmp_path / ("rank%d.json" % r)))["max"] == 2.5


def test_reference_arm_under_torchrun_two_ranks():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1          # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    # the rest of the line's contract: same keys as the GPU arm, the CPU run
    # described, no host-device bytes
    for k in ("metric", "unit", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
              "dtype", "data", "config", "e2e"):
        assert k in d, k
    assert d["steps"] == 1 and d["warmup"] == 3 and "workload" in d["config"]
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def _part_main(rank, world, port, out_dir):
    """One rank of a row-partitioned KPM-DOS run over gloo: its z-slab of
    the lattice, the CPU local step, the halo exchanged with the other rank
    before every sweep and the scalar products summed once at the end."""
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import torch.distributed as dist
    from kpm_inputs import hamiltonians as ham
    from oracle import oracle
    from paper_1410_5242_gb300 import partition
    from part_cpu_step import CpuPartStep
    dist.init_process_group("gloo")
    h = ham.ti_hamiltonian(4, 3, 6, gamma=0.8, seed=4)
    a, b = oracle.scale_from_bounds(*oracle.gershgorin(h), 0.01)
    rs = partition.slab_row_start(h["n"], world, plane_rows=4 * 3 * 4)
    part = partition.build_parts(h, rs)[rank]
    eta, eti = partition.part_moments(CpuPartStep(part, a, b), partition.TorchComm(), 40, 3, 7)
    np.save(os.path.join(out_dir, "eta%d.npy" % rank), eta)
    np.save(os.path.join(out_dir, "eti%d.npy" % rank), eti)
    dist.destroy_process_group()


def test_row_partitioned_run_over_gloo_matches_the_oracle(tmp_path, orc):
    import numpy as np
    import torch.multiprocessing as mp
    from kpm_inputs import hamiltonians as ham
    port = free_port()
    mp.spawn(_part_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    h = ham.ti_hamiltonian(4, 3, 6, gamma=0.8, seed=4)
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    ref, _ = orc.moments(h, a, b, 40, 7, range(3))
    etas = [np.load(tmp_path / ("eta%d.npy" % r)) for r in range(2)]
    assert np.array_equal(etas[0], etas[1])  # one all-reduce: every rank holds the same sums
    assert np.all(np.abs(etas[0] - ref) <= 1e-10 * ref[:, :1])
    assert np.all(np.abs(np.load(tmp_path / "eti0.npy")) <= 1e-12 * ref[:, :1])
