"""Randomized planner check on the CPU: seeded random circuits (all ten gate
types, sparse two-qubit structure with lone qubits, Hadamard and RZ layers)
under random planner options (planner, |A| limit, fused width, precision,
forced low qubits, pruning threshold, attachment, staging).  Every plan must
build, pass the library's and the oracle's validity checks, and -- applied
kernel by kernel through the FP64 fused unitaries and the program emulator,
staged plans on their chunk views -- reproduce the FP64 oracle."""
import numpy as np
import pytest

from oracle import plan as OP
from oracle import sim
from synth import circuits as C
from tests.program_emulator import run_any_plan

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")


def _circuit(rng, n):
    kind = int(rng.integers(0, 5))
    lone = set(rng.choice(n, size=int(rng.integers(0, max(1, n // 2))), replace=False).tolist()) if kind in (1, 2) else set()
    pool = [q for q in range(n) if q not in lone] or list(range(n))
    items = []
    for _ in range(int(rng.integers(0, 100))):
        t = int(rng.integers(0, 10))
        th = list(rng.uniform(0, 2 * np.pi, size=C.NPARAM[t]))
        if C.NQ[t] == 2:
            if len(pool) >= 2:
                a, b = rng.choice(pool, size=2, replace=False)
                items.append((t, int(a), int(b), *th))
        else:
            items.append((t, int(rng.integers(0, n)), None, *th))
    if kind == 3:
        items = [(C.H, q, None) for q in range(n)] + items
    if kind == 4:
        items = items + [(C.RZ, q, None, 0.3) for q in range(n)]
    return C.make_gates(items)


@pytest.mark.parametrize("seed", range(3))
def test_random_circuits_and_options(seed):
    rng = np.random.default_rng(1000 + seed)
    checked = 0
    for it in range(30):
        n = int(rng.integers(10, 14))
        g = _circuit(rng, n)
        kw = dict(algo=int(rng.choice([1, 2, 3])), shm_max_active=int(rng.integers(6, 15)),
                  fuse_kmax=int(rng.choice([0, 2, 4, 6])), precision=int(rng.choice([0, 0, 2])),
                  forced_low=int(rng.choice([0, 2, 4])), prune_T=int(rng.choice([16, 64, 500])),
                  attach_single=int(rng.choice([0, 1])), shm_variant=2)
        kw["forced_low"] = min(kw["forced_low"], kw["shm_max_active"])
        if rng.uniform() < 0.3 and n >= 13:
            kw["local_qubits"] = int(rng.integers(12, n))
            kw["shm_max_active"] = min(kw["shm_max_active"], kw["local_qubits"])
        try:
            p = Q.Plan(n, g, **kw)
        except Q.QsError as e:
            # tensor-core widths need n >= 11; a staged plan needs L >= 12 and
            # L >= |A| and forced low + 2: option combinations the API refuses
            assert e.status in (Q.QS_EUNSUPPORTED, Q.QS_EINVAL), (it, kw, e)
            continue
        assert p.validate() == 0, (it, kw)
        OP.check_plan(g, p.kernels())
        psi0 = np.random.default_rng(it).normal(size=1 << n) + 0j
        psi0 /= np.linalg.norm(psi0)
        got = run_any_plan(p, n, psi0.copy())
        if got is None:
            continue
        ref = sim.apply(n, g, psi0.copy())
        assert np.max(np.abs(got - ref)) <= 1e-5, (it, kw)
        checked += 1
    assert checked >= 15


def test_planning_at_larger_sizes():
    # 17 to 30 qubits, the benchmark families and random circuits, staged or
    # not: every plan builds and is valid by the library and by the oracle
    rng = np.random.default_rng(2024)
    for it in range(12):
        n = int(rng.integers(17, 31))
        fam = it % 4
        g = [lambda: C.mixed_circuit(n, int(rng.integers(100, 1500)), it),
             lambda: C.entangling_circuit(n, int(rng.integers(1, 12)), it),
             lambda: C.layered_u3_cz(n, int(rng.integers(1, 12)), it),
             lambda: _circuit(rng, n)][fam]()
        kw = dict(algo=int(rng.choice([1, 2, 3])), shm_max_active=int(rng.integers(8, 15)),
                  fuse_kmax=int(rng.choice([0, 4, 6])), precision=int(rng.choice([0, 2])),
                  forced_low=int(rng.choice([2, 4])), prune_T=int(rng.choice([16, 100])), shm_variant=1)
        if it % 3 == 0:
            kw["local_qubits"] = int(rng.integers(max(12, kw["shm_max_active"]), n))
            kw["stager"] = int(rng.choice([0, 1]))
        p = Q.Plan(n, g, **kw)
        assert p.validate() == 0
        OP.check_plan(g, p.kernels())
