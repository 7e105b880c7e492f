"""Placement of simulations on devices by HBM budget (apic_place_by_budget),
on the CPU: the rule itself, the balance it gives a stream of admissions,
and two gloo ranks reaching the same partition of a simulation list with no
exchange of data (the rule is deterministic)."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BIG = 2**63 - 1


@pytest.fixture(scope="module")
def apic():
    from paper_2108_02259_gb300 import apic, build

    build.build()
    return apic


def test_rule(apic):
    place = apic.place_by_budget
    assert place([10, 30, 20], 5) == 1          # the most room
    assert place([30, 30, 20], 5) == 0          # ties: the lowest index
    assert place([10, 30, 20], 25) == 1
    assert place([10, 30, 20], 31) == -1        # nothing holds it
    assert place([10, BIG, 20], 10**15) == 1    # a device without a budget
    assert place([0, 0], 0) == 0                # an empty simulation fits anywhere
    assert place([5], -1) == -1                 # a negative size is refused


def greedy_partition(apic, sizes, budgets):
    """Admit sizes in order with the group's rule; returns the member of each
    (or -1) and the bytes left per member."""
    room = list(budgets)
    out = []
    for s in sizes:
        k = apic.place_by_budget(room, s)
        out.append(k)
        if k >= 0:
            room[k] -= s
    return out, room


def test_stream_of_admissions_stays_balanced(apic):
    """With room for everything, the members' loads never differ by more
    than the largest simulation (each goes where the most room is left)."""
    rng = np.random.default_rng(3)
    sizes = [int(s) for s in np.exp(rng.uniform(np.log(2e3), np.log(1e6), 256)) * 2000]
    for n_dev in (2, 3, 4, 8):
        budget = 2 * sum(sizes)
        member, room = greedy_partition(apic, sizes, [budget] * n_dev)
        assert min(member) >= 0
        loads = [budget - r for r in room]
        assert max(loads) - min(loads) <= max(sizes)
        assert sum(loads) == sum(sizes)


def test_refusal_when_no_member_has_room(apic):
    sizes = [60, 50, 40, 30]
    member, room = greedy_partition(apic, sizes, [100, 70])
    assert member == [0, 1, 0, -1]
    assert room == [0, 20]


def _rank_main(rank, ws, port, out_dir):
    import json
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2108_02259_gb300 import apic

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    rng = np.random.default_rng(11)  # the same simulation list on every rank
    sizes = [int(s) for s in np.exp(rng.uniform(np.log(2e3), np.log(1e6), 200)) * 2000]
    member, _ = greedy_partition(apic, sizes, [2 * sum(sizes)] * ws)
    mine = [i for i, k in enumerate(member) if k == rank]  # what this rank would admit on its device
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"member": member, "mine": mine}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_partition(tmp_path):
    import json

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["member"] == r1["member"]
    assert sorted(r0["mine"] + r1["mine"]) == list(range(200))  # every simulation on exactly one rank
    assert not set(r0["mine"]) & set(r1["mine"])
