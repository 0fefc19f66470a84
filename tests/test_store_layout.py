"""CPU check of the register-phased programs' global-memory layout: the load
phase keeps local bits 0..3 (the forced low qubits) on lanes 0..3, so each
group of four lanes reads one 128-B run, and the store phase keeps local
bits 0 and 1 on lanes 0 and 1, so each group of four lanes writes one whole
32-B sector (QSIM_STORE_SECTORS=0: bits 0..3, whole 128-B runs).  The maps
are read from the programs' exchange words (PK_XCHG carries the new phase's
thread bits) and, for the load phase, from the first exchange's inverse
view: every local bit that is not a register slot of the load phase is a
thread bit."""
import numpy as np
import pytest

from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")
SZ = {1: 9, 2: 5, 3: 5, 4: 9, 5: 1, 6: 1, 7: 1, 8: 5, 9: 3, 10: 9, 11: 9, 12: 3, 13: 9, 14: 1, 15: 3, 16: 3, 18: 33}
PK_END, PK_XCHG = 0, 17


def _maps(words):
    """Thread-bit lists (lane order) of every phase after the load phase."""
    out, pc = [], 0
    while pc < len(words):
        op = int(words[pc]) & 0xFF
        if op == PK_END:
            break
        if op == PK_XCHG:
            nt = (int(words[pc]) >> 8) & 0xFF
            regs = [int(w).bit_length() - 1 for w in words[pc + 1:pc + 6]]
            lanes = [(int(w) & 0xFFFF).bit_length() - 1 for w in words[pc + 6:pc + 6 + nt]]
            out.append((regs, lanes))
            pc += 6 + nt
            continue
        pc += SZ[op]
    return out


@pytest.mark.parametrize("sectors", ["1", "0"])
@pytest.mark.parametrize("kind", ["mixed", "entangling", "layered"])
def test_store_phase_lanes(kind, sectors, monkeypatch):
    monkeypatch.setenv("QSIM_STORE_SECTORS", sectors)
    n = 16
    g = {"mixed": C.mixed_circuit(n, 600, 5), "entangling": C.entangling_circuit(n, 6, 5),
         "layered": C.layered_u3_cz(n, 8, 5)}[kind]
    plan = Q.Plan(n, g, algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=12, forced_low=4)
    need = 2 if sectors == "1" else 4
    stores_in_sectors = 0
    for k in range(plan.stats().num_kernels):
        words, m, act, R = plan.kernel_program(k)
        assert act[:4] == [0, 1, 2, 3]  # the forced low qubits are local bits 0..3
        assert not set(R) & {0, 1, 2, 3}  # load phase: low bits on lanes
        maps = _maps(words)
        if not maps:
            continue
        regs, lanes = maps[-1]
        assert lanes[:need] == list(range(need)), (k, regs, lanes)
        assert not set(regs) & set(range(need))
        stores_in_sectors += bool(set(regs) & {2, 3})
    if sectors == "0":
        assert stores_in_sectors == 0
    elif kind == "mixed":
        assert stores_in_sectors > 0  # the rule is exercised: some kernel stores from bit 2 or 3
