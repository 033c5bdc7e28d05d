"""Serving loop (GPU): continuous batching over device-resident systems of different grid, atom, band
and numax sizes.  A request's result is the same alone and in the mix (bitwise: every kernel is
deterministic and each request works on its own system's buffers), the served result equals the
direct entry point and the oracle, admission respects the memory budget, waits are bounded."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _systems(count, seed=77):
    import torch
    rng = np.random.default_rng(seed)
    out = []
    specs = [(48, 8, 16, 3), (64, 20, 48, 5), (48, 12, 32, 7), (80, 30, 16, 9), (64, 16, 64, 5), (48, 24, 32, 3)]
    for i in range(count):
        g, na, nb, nu = specs[i % len(specs)]
        pos, sig = workloads.random_atoms(rng, na, (g * 0.2,) * 3, True, min_sep=1.5)
        psi = torch.from_numpy(rng.standard_normal((g, g, g, nb)).astype(np.float32)).cuda()
        out.append(dict(psi=psi, pos=pos, sig=sig, numax=nu, cube=32, h=0.2))
    return out


def _run(server, systems, ops, concurrent):
    ids = [server.register(s["psi"], s["pos"], s["sig"], s["numax"], s["cube"], s["h"]) for s in systems]
    tickets = []
    if concurrent:
        for op in ops:
            for sid in ids:
                tickets.append(server.submit(sid, op, "fp32"))
        for t in tickets:
            assert server.wait(t, 120000) == 0
    else:
        for sid in ids:
            for op in ops:
                assert server.wait(server.submit(sid, op, "fp32"), 120000) == 0
    res = [server.read(sid) for sid in ids]
    for sid in ids:
        server.unregister(sid)
    return res


def test_alone_equals_mix_and_direct_and_oracle():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    from paper_1905_00480_gb300.serve import Server
    systems = _systems(6)
    with Server(0, budget_bytes=16 << 30, slots=4) as srv:
        alone = _run(srv, systems, ["project", "expand"], concurrent=False)
        mix = _run(srv, systems, ["project", "expand"], concurrent=True)
        st = srv.stats()
    assert st["max_inflight"] >= 2, "requests of different systems should overlap"
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for (pa, ca), (pm, cm) in zip(alone, mix):
        assert torch.equal(pa, pm) and torch.equal(ca, cm)
    # served project == direct entry point (same kernels): bitwise
    s0 = systems[1]
    c = api.project(s0["psi"], s0["pos"], s0["sig"], s0["numax"], 32, 0.2, True, prec="fp32")
    assert torch.equal(c.cpu(), alone[1][1])
    # and the oracle within the FP32 tolerance
    ref = oracle.project((64,) * 3, 0.2, True, s0["psi"].double().cpu().numpy(), s0["pos"], s0["sig"], 5, 32)
    assert rel_norm(alone[1][1].double().numpy(), ref) <= TOL_FP32
    # the served expansion (psi += E c with c the served projection) against the oracle expansion
    psi_in = s0["psi"].double().cpu().numpy()
    ref_add = oracle.add((64,) * 3, 0.2, True, np.zeros_like(psi_in), s0["pos"], s0["sig"], 5, 32,
                         alone[1][1].double().numpy())
    assert rel_norm(alone[1][0].double().numpy() - psi_in, ref_add) <= TOL_FP32
    for k in (0, 2, 5):   # other sizes and numax 3 / 7 / 3
        sk = systems[k]
        g = sk["psi"].shape[0]
        pin = sk["psi"].double().cpu().numpy()
        refc = oracle.project((g,) * 3, 0.2, True, pin, sk["pos"], sk["sig"], sk["numax"], 32)
        assert rel_norm(alone[k][1].double().numpy(), refc) <= TOL_FP32
        refa = oracle.add((g,) * 3, 0.2, True, np.zeros_like(pin), sk["pos"], sk["sig"], sk["numax"], 32,
                          alone[k][1].double().numpy())
        assert rel_norm(alone[k][0].double().numpy() - pin, refa) <= TOL_FP32


def test_admission_respects_budget():
    """Resident systems plus in-flight workspaces never exceed the budget; with room, requests of
    different systems overlap."""
    require_gpu()
    from paper_1905_00480_gb300.serve import Server
    systems = _systems(3, seed=5)[:3]
    resident = sum(s["psi"].numel() * 4 for s in systems) + sum(
        len(s["pos"]) * oracle.nstates(s["numax"]) * s["psi"].shape[3] * 4 for s in systems)
    # the largest expansion workspace of these systems (the z-pass intermediate dominates: FP32, stored
    # band-tiled [A][cube][B/32][32][PP] for the block gather, PP = pairs rounded up to 4, plus 4 when
    # that is a multiple of 8), plus plan slack
    def t2_bytes(s):
        P = (s["numax"] + 1) * (s["numax"] + 2) // 2
        PP = (P + 3) // 4 * 4
        PP += 4 if PP % 8 == 0 else 0
        B = s["psi"].shape[3]
        return len(s["pos"]) * 32 * max(P * B, (B + 31) // 32 * 32 * PP) * 4
    need = max(t2_bytes(s) for s in systems)
    budget = resident + need + (1 << 20)
    with Server(0, budget_bytes=budget, slots=4) as srv:
        _run(srv, systems, ["expand", "expand"], concurrent=True)
        tight = srv.stats()
    assert tight["completed"] == 6 and tight["failed"] == 0
    assert tight["peak_bytes"] <= budget
    with Server(0, budget_bytes=8 << 30, slots=4) as srv:
        _run(srv, systems, ["expand", "expand"], concurrent=True)
        roomy = srv.stats()
    assert roomy["completed"] == 6 and roomy["max_inflight"] >= 2


def test_capacity_and_state_errors():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import ShoError
    from paper_1905_00480_gb300.serve import Server
    psi = torch.zeros((48, 48, 48, 16), dtype=torch.float32, device="cuda")
    with Server(0, budget_bytes=1 << 20, slots=2) as srv:
        with pytest.raises(ShoError, match="CAPACITY"):
            srv.register(psi, np.array([[4.0, 4.0, 4.0]]), [0.7], 3, 32, 0.2)
    with Server(0, budget_bytes=1 << 30, slots=2) as srv:
        with pytest.raises(ShoError, match="STATE"):
            srv.submit(12345, "project")


def test_wait_is_bounded():
    """A wait with a zero timeout on a running request returns a timeout (host side; the request keeps
    running and completes)."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300.serve import Server
    rng = np.random.default_rng(3)
    pos, sig = workloads.random_atoms(rng, 200, (19.2,) * 3, True, min_sep=1.2)
    psi = torch.randn((96, 96, 96, 128), dtype=torch.float32, device="cuda")
    with Server(0, budget_bytes=8 << 30, slots=2) as srv:
        sid = srv.register(psi, pos, sig, 9, 32, 0.2)
        t = srv.submit(sid, "project", "fp32")
        with pytest.raises(TimeoutError):
            srv.wait(t, 0)
        assert srv.wait(t, 120000) == 0
