"""Continuous batching: a right-hand side solved alone and in the mix gives the same field.

The mixed run submits other sources first, steps the server so they are in flight, then submits
the probe source, which joins at a later FGMRES iteration; every result must match the oracle's
global solve to 1e-6 and the probe must equal its solo result to 1e-6.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.discretize import Problem, extend_interior, rhs_from_source
from oracle.linsolve import global_solve
from paper_2003_02585_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_server_result_alone_equals_result_in_the_mix():
    from paper_2003_02585_gb300 import dds
    n = (96, 96)
    h = 1.0 / 96
    c = synth.medium_two_layer(n, h)
    kappa = 2 * np.pi * 6
    ctx = dds.Context(n, h, kappa, c, (3, 3), 10, 30.0, precision="mixed")
    prob = Problem(n, h, kappa, c, (3, 3), 10, 30.0)
    centres = [(0.3, 0.7), (0.6, 0.2), (0.5, 0.5), (0.8, 0.8)]
    f = ctx.extend(synth.gaussian_sources(n, h, centres, 2 * h))
    ug = global_solve(prob, rhs_from_source(prob, extend_interior(
        prob, synth.gaussian_sources(n, h, centres, 2 * h))))

    solo = dds.Server(ctx, 4, 1e-9, 30, 1)
    solo.submit(f[0], 0)
    res = None
    while res is None:
        solo.step()
        res = solo.poll()
    u_alone = res[1].copy()
    assert res[3] < 1e-9 and _rel(u_alone, ug[0]) < 1e-6

    mix = dds.Server(ctx, 3, 1e-9, 30, 1)
    mix.submit(f[1], 1)
    mix.submit(f[2], 2)
    active, _ = mix.step()
    assert active == 2
    mix.submit(f[0], 0)            # arrives while 1 and 2 are in flight
    mix.submit(f[3], 3)            # waits for a free slot (3 slots)
    got = {}
    overlap = False
    for _ in range(200):
        active, queued = mix.step()
        overlap |= active == 3
        while True:
            r = mix.poll()
            if r is None:
                break
            got[r[0]] = (r[1].copy(), r[2], r[3])
        if len(got) == 4:
            break
    assert overlap and sorted(got) == [0, 1, 2, 3]
    for k in range(4):
        assert got[k][2] < 1e-9
        assert _rel(got[k][0], ug[k]) < 1e-6
    assert _rel(got[0][0], u_alone) < 1e-6


def test_server_admits_by_device_memory():
    """dds_server_create takes as many slots as the context's budget leaves room for (at most
    max_slots): a larger budget admits more slots, a budget with no room for one slot is
    DDS_ENOMEM, and the slots a server holds count against the budget."""
    from paper_2003_02585_gb300 import dds
    n = (96, 96)
    h = 1.0 / 96
    ctx = dds.Context(n, h, 2 * np.pi * 6, synth.medium_constant(n), (3, 3), 10, 30.0,
                      precision="mixed")
    held = ctx.info()["device_bytes"]
    field = 16 * int(np.prod(ctx.G))
    per_slot_floor = field * (2 * 20 + 5)          # the basis and batch fields alone
    ctx.set_memory_budget(held + 3 * per_slot_floor)
    s_small = dds.Server(ctx, 64, 1e-6, 20, 1)
    assert 1 <= s_small.slots <= 3
    assert ctx.info()["device_bytes"] <= held + 3 * per_slot_floor
    s_small.close()
    ctx.set_memory_budget(held + 12 * per_slot_floor)
    s_big = dds.Server(ctx, 64, 1e-6, 20, 1)
    assert s_small.slots < s_big.slots <= 12
    s_big.close()
    ctx.set_memory_budget(held + per_slot_floor // 4)
    with pytest.raises(dds.DDSError) as e:
        dds.Server(ctx, 64, 1e-6, 20, 1)
    assert e.value.status == 2                     # DDS_ENOMEM
    ctx.set_memory_budget(0)
    assert dds.Server(ctx, 5, 1e-6, 20, 1).slots == 5


def test_budgeted_server_steps_batches_of_every_size():
    """A server created under a tight budget still has room, at every step, for what a step
    allocates besides its slots (the DDM plan of each new batch size): requests arriving one, two
    and three at a time all finish without DDS_ENOMEM, each to the tolerance."""
    from paper_2003_02585_gb300 import dds
    n = (96, 96)
    h = 1.0 / 96
    ctx = dds.Context(n, h, 2 * np.pi * 6, synth.medium_two_layer(n, h), (3, 3), 10, 30.0,
                      precision="mixed", plan="trace")
    held = ctx.info()["device_bytes"]
    field = 16 * int(np.prod(ctx.G))
    ctx.set_memory_budget(held + 8 * field * (2 * 12 + 5))
    srv = dds.Server(ctx, 64, 1e-6, 12, 2)
    assert srv.slots >= 3
    rng = np.random.default_rng(7)
    tag = 0
    done = []
    for burst in (1, 2, 3, srv.slots, 1):
        for _ in range(burst):
            f = synth.gaussian_sources(n, h, [tuple(rng.uniform(0.2, 0.8, size=2))], 2 * h)
            srv.submit(ctx.extend(f), tag)
            tag += 1
        for _ in range(200):
            active, queued = srv.step()
            while (r := srv.poll()) is not None:
                done.append(r)
            if active == 0 and queued == 0:
                break
    assert len(done) == tag
    assert max(r[3] for r in done) <= 1e-6
    srv.close()


def test_sources_waiting_beyond_the_budget_queue_in_host_memory():
    """More sources than the budget holds device copies for are all accepted (the overflow waits
    in host memory) and all solved, each to the tolerance."""
    from paper_2003_02585_gb300 import dds
    n = (96, 96)
    h = 1.0 / 96
    ctx = dds.Context(n, h, 2 * np.pi * 6, synth.medium_constant(n), (3, 3), 10, 30.0,
                      precision="mixed")
    held = ctx.info()["device_bytes"]
    field = 16 * int(np.prod(ctx.G))
    floor = field * (2 * 12 + 5)                  # one slot's basis and batch fields
    budget = held + (5 * floor) // 2              # two slots at most, and about ten spare fields
    ctx.set_memory_budget(budget)
    srv = dds.Server(ctx, 2, 1e-6, 12, 1)
    rng = np.random.default_rng(11)
    nreq = 40                                     # far more waiting fields than the budget's room
    for tag in range(nreq):
        f = synth.gaussian_sources(n, h, [tuple(rng.uniform(0.2, 0.8, size=2))], 2 * h)
        srv.submit(ctx.extend(f), tag)
    assert ctx.info()["device_bytes"] <= budget
    done = []
    for _ in range(2000):
        active, queued = srv.step()
        while (r := srv.poll()) is not None:
            done.append(r)
        if active == 0 and queued == 0:
            break
    assert sorted(r[0] for r in done) == list(range(nreq))
    assert max(r[3] for r in done) <= 1e-6
    srv.close()


def test_context_destroyed_before_its_server():
    """A server may outlive its context (garbage collection can finalise them in any order): the
    context's destruction releases the server's device memory, later calls on the server are
    rejected with DDS_EINVAL, and destroying the server afterwards is safe."""
    from paper_2003_02585_gb300 import dds
    n = (48, 48)
    h = 1.0 / 48
    ctx = dds.Context(n, h, 2 * np.pi * 3, synth.medium_constant(n), (2, 2), 6, 30.0,
                      precision="mixed")
    srv = dds.Server(ctx, 4, 1e-6, 10, 1)
    f = synth.gaussian_sources(n, h, [(0.4, 0.6)], 2 * h)
    srv.submit(ctx.extend(f), 1)
    srv.step()
    ctx.close()
    with pytest.raises(dds.DDSError) as e:
        srv.step()
    assert e.value.status == 1                     # DDS_EINVAL
    srv.close()
