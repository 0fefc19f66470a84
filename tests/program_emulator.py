"""A plain numpy emulator of the register-phased shared-memory programs
(opcodes of shm_program.hpp), for CPU tests of the program compiler.

It executes a program's words by their documented meaning on complex128
tiles, for every batch of the kernel at once: register slot i denotes local
bit R[i] of the current phase (an exchange only changes R), a known-bit
reference denotes a thread bit of the local index or a batch (non-active)
qubit.  It shares nothing with the CUDA kernels but the program format."""
import numpy as np

PK_END, PK_G1, PK_G1R, PK_G1X, PK_G1C, PK_XG, PK_XGS, PK_XGK = 0, 1, 2, 3, 4, 5, 6, 7
PK_D1, PK_D1B, PK_D1K, PK_D2, PK_D2P, PK_D0, PK_SWAPR, PK_XX = 8, 9, 10, 11, 12, 13, 14, 15
PK_SCALE, PK_XCHG, PK_G2 = 16, 17, 18
REF_NONE, REF_LOCAL, REF_GLOBAL = 0xFF, 0x40, 0x80
NSLOTS = 5


def _f(words, i):
    return float(np.array([words[i]], dtype=np.uint32).view(np.float32)[0])


def _c(words, i):
    return complex(_f(words, i), _f(words, i + 1))


def run_kernel(psi, n, words, m, act, R0):
    """Applies one kernel's program to psi (complex128, length 2^n) in place."""
    act = list(act)
    li = np.arange(1 << m, dtype=np.int64)
    phys = np.zeros(1 << m, dtype=np.int64)
    for j, q in enumerate(act):
        phys |= ((li >> j) & 1) << q
    nonact = [q for q in range(n) if q not in act]
    b = np.arange(1 << (n - m), dtype=np.int64)
    base = np.zeros_like(b)
    for k, q in enumerate(nonact):
        base |= ((b >> k) & 1) << q
    tile = psi[base[:, None] | phys[None, :]]  # (batches, 2^m)
    R = list(R0)

    def lbit(slot):
        return R[slot]

    def known(ref):  # 0/1 array broadcastable to the tile
        if ref & REF_GLOBAL:
            return ((base >> (ref & 63)) & 1)[:, None]
        return ((li >> (ref & 31)) & 1)[None, :]

    def pairs(slot):
        lb = lbit(slot)
        lo = li[((li >> lb) & 1) == 0]
        return lo, lo | (1 << lb)

    def apply2(slot, u00, u01, u10, u11, ctrl=None):
        # ctrl: 0/1 array broadcastable to the tile; the pair is updated where
        # it is 1 (a control bit differs from the target bit, so the pair's
        # two amplitudes agree on it)
        lo, hi = pairs(slot)
        x, y = tile[:, lo].copy(), tile[:, hi].copy()
        nx, ny = u00 * x + u01 * y, u10 * x + u11 * y
        if ctrl is not None:
            c = np.broadcast_to(ctrl, tile.shape)[:, lo] == 1
            nx, ny = np.where(c, nx, x), np.where(c, ny, y)
        tile[:, lo], tile[:, hi] = nx, ny

    pc = 0
    while True:
        w = int(words[pc])
        op, A, B, Cu = w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 0xFF, w >> 24
        if op == PK_END:
            break
        if op == PK_G1:
            apply2(A, _c(words, pc + 1), _c(words, pc + 3), _c(words, pc + 5), _c(words, pc + 7))
            pc += 9
        elif op == PK_G1R:
            apply2(A, _f(words, pc + 1), _f(words, pc + 2), _f(words, pc + 3), _f(words, pc + 4))
            pc += 5
        elif op == PK_G1X:
            apply2(A, _f(words, pc + 1), 1j * _f(words, pc + 2), 1j * _f(words, pc + 3), _f(words, pc + 4))
            pc += 5
        elif op == PK_G1C:
            ctrl = ((li >> lbit(B)) & 1)[None, :] if B < NSLOTS else known(B)
            apply2(A, _c(words, pc + 1), _c(words, pc + 3), _c(words, pc + 5), _c(words, pc + 7), ctrl)
            pc += 9
        elif op in (PK_XG, PK_XGS, PK_XGK):
            lo, hi = pairs(A)
            if op == PK_XGS:
                sel = ((lo >> lbit(B)) & 1) == 1
                lo, hi = lo[sel], hi[sel]
                tile[:, lo], tile[:, hi] = tile[:, hi].copy(), tile[:, lo].copy()
            elif op == PK_XGK:
                apply2(A, 0.0, 1.0, 1.0, 0.0, known(B))
            else:
                tile[:, lo], tile[:, hi] = tile[:, hi].copy(), tile[:, lo].copy()
            pc += 1
        elif op == PK_D1:
            bit = (li >> lbit(A)) & 1
            tile *= np.where(bit == 1, _c(words, pc + 3), _c(words, pc + 1))[None, :]
            pc += 5
        elif op == PK_D1B:
            bit = (li >> lbit(A)) & 1
            tile *= np.where(bit == 1, _c(words, pc + 1), 1.0)[None, :]
            pc += 3
        elif op == PK_D1K:
            d = [_c(words, pc + 1 + 2 * e) for e in range(4)]
            bit = ((li >> lbit(A)) & 1)[None, :]
            idx = bit + 2 * known(B)
            tile *= np.asarray(d)[idx]
            pc += 9
        elif op == PK_D2:
            d = np.asarray([_c(words, pc + 1 + 2 * e) for e in range(4)])
            idx = ((li >> lbit(A)) & 1) + 2 * ((li >> lbit(B)) & 1)
            tile *= d[idx][None, :]
            pc += 9
        elif op == PK_D2P:
            both = (((li >> lbit(A)) & 1) & ((li >> lbit(B)) & 1)) == 1
            tile *= np.where(both, _c(words, pc + 1), 1.0)[None, :]
            pc += 3
        elif op == PK_D0:
            d = np.asarray([_c(words, pc + 1 + 2 * e) for e in range(4)])
            idx = known(A) + (0 if B == REF_NONE else 2 * known(B))
            unit = np.asarray([(Cu >> e) & 1 for e in range(4)])
            f = np.where(unit[idx] == 1, 1.0, d[idx])
            tile *= f
            pc += 9
        elif op == PK_SWAPR:
            la, lb = lbit(A), lbit(B)
            src = li[(((li >> la) & 1) == 1) & (((li >> lb) & 1) == 0)]
            dst = src ^ (1 << la) ^ (1 << lb)
            tile[:, src], tile[:, dst] = tile[:, dst].copy(), tile[:, src].copy()
            pc += 1
        elif op == PK_XX:
            c, s = _f(words, pc + 1), _f(words, pc + 2)
            la, lb = lbit(A), lbit(B)
            j = li[((li >> lb) & 1) == 0]
            k = j ^ (1 << la) ^ (1 << lb)
            x, y = tile[:, j].copy(), tile[:, k].copy()
            tile[:, j] = c * x - 1j * s * y
            tile[:, k] = c * y - 1j * s * x
            pc += 3
        elif op == PK_SCALE:
            tile *= _c(words, pc + 1)
            pc += 3
        elif op == PK_XCHG:
            nt = A
            R = [int(words[pc + 1 + i]).bit_length() - 1 for i in range(NSLOTS)]
            pc += 1 + NSLOTS + nt
        elif op == PK_G2:
            g = np.asarray([_c(words, pc + 1 + 2 * e) for e in range(16)]).reshape(4, 4)
            la, lb = lbit(A), lbit(B)
            j = li[(((li >> la) & 1) == 0) & (((li >> lb) & 1) == 0)]
            idx = [j, j | (1 << la), j | (1 << lb), j | (1 << la) | (1 << lb)]
            x = [tile[:, t].copy() for t in idx]
            for r in range(4):
                tile[:, idx[r]] = sum(g[r, k] * x[k] for k in range(4))
            pc += 33
        else:
            raise ValueError(f"unknown opcode {op} at word {pc}")
    psi[base[:, None] | phys[None, :]] = tile


def run_plan(plan, n, psi):
    """Applies every kernel of an all-shared-memory plan to psi in place."""
    for k in range(plan.stats().num_kernels):
        words, m, act, R = plan.kernel_program(k)
        run_kernel(psi, n, words, m, act, R)
    return psi


def apply_unitary(psi, n, qubits, u):
    """psi <- u on the given qubits (index bit j of u's rows and columns is
    qubits[j]): gather, matrix product, scatter."""
    k = len(qubits)
    sub = np.zeros(1 << k, dtype=np.int64)
    for j, q in enumerate(qubits):
        sub |= ((np.arange(1 << k) >> j) & 1) << q
    rest = [q for q in range(n) if q not in qubits]
    base = np.zeros(1 << (n - k), dtype=np.int64)
    for j, q in enumerate(rest):
        base |= ((np.arange(1 << (n - k)) >> j) & 1) << q
    idx = base[:, None] | sub[None, :]
    psi[idx] = psi[idx] @ u.T


def run_any_plan(plan, n, psi, fused_kernel_type=1):
    """Applies any plan (fused kernels by their FP64 unitaries, shared-memory
    kernels by their programs; a staged plan stage by stage on its chunk
    view) to psi in place.  Returns None when a shared-memory kernel has no
    register-phased program."""
    L = plan.opts.local_qubits
    stats = plan.stats()
    if 0 < L < n:
        idx = np.arange(1 << n)
        views = []
        for si in range(stats.num_stages):
            st = plan.stage(si)
            local = [q for q in range(n) if (st["local_mask"] >> q) & 1]
            order = local + [q for q in range(n) if not (st["local_mask"] >> q) & 1]
            logical = np.zeros_like(idx)
            for p, q in enumerate(order):
                logical |= ((idx >> p) & 1) << q
            views.append((logical, {q: p for p, q in enumerate(order)},
                          range(st["first_kernel"], st["first_kernel"] + st["num_kernels"])))
    else:
        views = [(None, {q: q for q in range(n)}, range(stats.num_kernels))]
    for logical, pos, kernels in views:
        view = psi if logical is None else psi[logical]
        for k in kernels:
            d = plan.kernel(k)
            if d.type == fused_kernel_type:
                apply_unitary(view, n, [pos[q] for q in range(n) if (d.qubit_mask >> q) & 1], plan.fused_matrix(k))
            else:
                try:
                    words, m, act, R = plan.kernel_program(k)
                except Exception:
                    return None
                run_kernel(view, n, words, m, act, R)
        if logical is not None:
            psi[logical] = view
    return psi
