"""Host logic of bench.py without a GPU: the max-over-ranks reduction of the
multi-rank (torchrun, one replica per rank) path on two gloo ranks, the
whole-job rate, and the reference arm's JSON line (the oracle on every
host core, one spawned process each; other ranks exit without output)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        # rank 0 is slower in the first value, rank 1 in the second
        got = bench.reduce_max([10.0 - rank, 3.0 + rank], 2)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump(got, f)
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            assert json.load(f) == [10.0, 4.0]


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([1.5, 2], 1) == [1.5, 2.0]


def test_whole_job_rate_is_weak_scaling():
    sys.path.insert(0, ROOT)
    import bench
    # 589824 updates per rank per step, 10 steps, 4 ranks, 2 ms
    assert bench.whole_job_rate(589824, 10, 4, 2e-3) == pytest.approx(589824 * 10 * 4 / 2e-3 / 1e9)


def test_hbm_view_of_a_form():
    """The dominant kernel with a byte count for the form, its GB/s from
    bytes per unit x units per launch / mean launch time."""
    sys.path.insert(0, ROOT)
    import bench
    prof = {"d2q9m_stage1": (10, 2.0), "d2q9m_stage2": (10, 1.5), "other": (5, 9.0)}
    v = bench.hbm_view(prof, "fp32", 9, 256, 256, 6800.0)
    want = 16 * 9 * 256 * 256 / (2.0e-3 / 10) / 1e9
    assert v["kernel"] == "d2q9m_stage1" and v["bytes_per_unit"] == 16
    assert v["achieved_gbs"] == pytest.approx(want) and v["frac"] == pytest.approx(want / 6800.0)
    # generic face kernels count face-velocities
    v = bench.hbm_view({"gdev_face_x": (2, 1.0)}, "bf16", 16, 10, 4, 1000.0)
    assert v["achieved_gbs"] == pytest.approx(6 * 16 * 4 * 11 / 0.5e-3 / 1e9)
    assert bench.hbm_view({"d2q9_stage1": (1, 1.0)}, "fp32", 9, 8, 8, 1.0) is None


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                           "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_arm_line():
    r = _run_reference({})
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "G updates/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["cpu_baseline"]["cpu_model"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "cavity256"


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
