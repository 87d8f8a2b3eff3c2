"""The N>1 form of the benchmark on CPU ranks (gloo, world size 2): every rank owns disjoint,
independent states (the REXI step of one state needs nothing from another, so the units are
sharded with no data-path collective), the job's time is the slowest rank's, and the
reference arm under torchrun prints one line from rank 0 while the other ranks exit 0."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import coeffs as oc  # noqa: E402
from oracle import rexi as orx  # noqa: E402
from paper_1805_06557_gb300 import synthetic as syn  # noqa: E402

T, N, DT, B = 7, 16, 3600.0, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _step_states(seeds):
    X = orx.spectrum_bound(T, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = bench.contour(X)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    return [orx.rexi_step(syn.gaussian_state(T, sd), T, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w)
            for sd in seeds]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.shard_seeds(rank, B)
    out = _step_states(seeds)          # this rank's units, no exchange with the other rank
    local_ms = 100.0 + 50.0 * rank     # rank 1 is the slower one
    value, max_ms = bench.job_rate(local_ms, B, world, 4, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, seeds, [o.tolist() for o in out], value, max_ms))


def test_two_ranks_shard_states_and_take_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    seeds = [s for r in res for s in r[1]]
    assert len(set(seeds)) == 2 * B                   # disjoint shards
    assert seeds == bench.shard_seeds(0, 2 * B)       # together: the job's states
    whole = _step_states(seeds)                       # one process over the whole job
    got = [np.array(o) for r in res for o in r[2]]
    for a, b in zip(got, whole):
        assert np.array_equal(a, b)
    for r in res:
        assert r[4] == 150.0                          # max over ranks
        assert abs(r[3] - B * 2 * 4 / 0.150) < 1e-9


def test_reference_arm_under_torchrun_rank0_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--T", "15",
           "--N", "32"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_orders_cover_the_step():
    """The reference arm's worker chunks hold every zonal order exactly once, with about equal
    work (T + 1 - m per order), so each timed step is a full step."""
    for t, parts in ((1, 4), (15, 3), (63, 16), (255, 16), (511, 7)):
        ch = bench._balanced_orders(t, parts)
        flat = sorted(m for c in ch for m in c)
        assert flat == list(range(t + 1))
        loads = [sum(t + 1 - m for m in c) for c in ch]
        assert max(loads) - min(loads) <= t + 1


# ---- the pole / zonal-order partition of one step (paper Sec. 5.3-5.4) -------------------------
TP, NP = 15, 64


def _partition_rank(rank, world, port, mode, q):
    """One rank of a partitioned step: its share by the library's host partition rule, computed
    by the oracle, completed by a sum all-reduce over gloo (the step that NCCL does on GPUs)."""
    import torch
    import torch.distributed as dist
    from paper_1805_06557_gb300 import rexi
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = orx.spectrum_bound(TP, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = bench.contour(X)
    z, w = oc.rexi_coefficients(NP, p0, Xc)
    U0 = syn.gaussian_state(TP, 11)
    own = rexi.partition(mode, TP, NP, rank, world)
    if mode == "poles":       # this rank's REXI terms: the sum over its poles only
        part = orx.rexi_step(U0, TP, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z[own], w[own])
    else:                     # this rank's zonal orders (the operator is block diagonal in m)
        mask = np.concatenate([np.full(TP + 1 - m, own[m]) for m in range(TP + 1)])
        part = orx.rexi_step(U0 * mask[None, :], TP, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w)
    t = torch.from_numpy(np.ascontiguousarray(part))
    dist.all_reduce(torch.view_as_real(t), op=dist.ReduceOp.SUM)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, own.tolist(), t.numpy().tolist()))


@pytest.mark.parametrize("mode", ["poles", "m"])
def test_two_ranks_partitioned_step_equals_whole_step(mode):
    """World size 2: every pole (conjugate pairs together) or zonal order is owned by exactly
    one rank, and the all-reduced sum of the ranks' shares equals the one-process step within
    FP64 summation-order rounding."""
    pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_rank, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    owns = np.array([r[1] for r in res])
    assert np.all(owns.sum(axis=0) == 1)                          # each unit on exactly one rank
    if mode == "poles":
        assert np.array_equal(owns[0], owns[0][::-1])             # conjugate pairs {k, N-1-k} whole
    else:
        cost = [sum(TP + 1 - m for m in range(TP + 1) if o[m]) for o in owns]
        assert abs(cost[0] - cost[1]) <= TP + 2                   # paired orders balance the chains
    X = orx.spectrum_bound(TP, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = bench.contour(X)
    z, w = oc.rexi_coefficients(NP, p0, Xc)
    whole = orx.rexi_step(syn.gaussian_state(TP, 11), TP, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w)
    for r in res:
        got = np.array(r[2])
        assert np.all(orx.rel_l2(got, whole, TP) < 1e-12)


def test_partition_rule_host():
    """rexi_partition: ownership is a partition for any world size; the large-weight poles (both
    ends of the node list) spread over the ranks; errors for bad arguments."""
    import __graft_entry__ as g
    g.build()
    from paper_1805_06557_gb300 import rexi
    for size in (1, 2, 3, 5):
        P = np.array([rexi.partition("poles", 255, 513, r, size) for r in range(size)])
        M = np.array([rexi.partition("m", 255, 513, r, size) for r in range(size)])
        assert np.all(P.sum(0) == 1) and np.all(M.sum(0) == 1)
        for r in range(size):
            assert np.array_equal(P[r], P[r][::-1])
        if size > 1:
            ends = P[:, :8].sum(1)                               # the 8 largest-weight nodes
            assert ends.max() - ends.min() <= 2
    with pytest.raises(rexi.RexiError):
        rexi.partition("poles", 15, 16, 2, 2)
