"""The traceback kernels' table layout and windowed walk, modelled on the CPU.

The kernels store one direction byte per band slot and anti-diagonal and walk
back through 32-row windows loaded into shared memory (kernel_tb.cuh).  This
test restates that geometry — the slot frame of each kernel (int32 lanes:
B(r) = ceil((r-w)/2), bytes in slot order; 16-bit lanes: floor((r-w)/2),
bytes 2p and 2p+1 of a lane from register p's halves), the window start and
width (80 bytes, or 144 for 24 slots per lane on 16-bit lanes, lane-aligned)
and both byte encodings — fills the tables from the band DP of the pins, and
checks that (1) every window load stays inside its pair's table, (2) every
byte the walk reads is a band cell's, and (3) the walk returns the oracle's
CIGAR.  It runs no GPU code: it pins the index arithmetic the kernels use.
"""
import numpy as np
import pytest

import pins
from oracle import oracle as O

NEG = -10**12

def ceil_div2(x):
    return -((-x) >> 1)


def dp_values(T, Q, p, w):
    """H,E,F,E2,F2 of every band cell (dict), oracle recurrences."""
    p = pins.normalise(p)
    tl, ql = len(T), len(Q)
    V = {}
    def get(t, q):
        if t == -1 and q == -1: return (0, NEG, NEG, NEG, NEG)
        if t == -1: return (-pins.gap(p, q + 1), NEG, NEG, NEG, NEG)
        if q == -1: return (-pins.gap(p, t + 1), NEG, NEG, NEG, NEG)
        return V.get((t, q), (NEG,) * 5)
    for t in range(tl):
        for q in range(ql):
            if abs(t - q) > w: continue
            hd = get(t - 1, q - 1)[0]
            if t == 0 and q > 0: hd = -pins.gap(p, q)
            if q == 0 and t > 0: hd = -pins.gap(p, t)
            up = get(t - 1, q); lf = get(t, q - 1)
            E = max(up[0] - p['q'] - p['e'], up[1] - p['e'])
            E2 = max(up[0] - p['q2'] - p['e2'], up[3] - p['e2'])
            F = max(lf[0] - p['q'] - p['e'], lf[2] - p['e'])
            F2 = max(lf[0] - p['q2'] - p['e2'], lf[4] - p['e2'])
            s = p['a'] if T[t] == Q[q] else -p['b']
            H = max(hd + s, E, F, E2, F2)
            V[(t, q)] = (H, E, F, E2, F2, hd + s)
    return V

def kernel_byte16(V, t, q, p):
    """The 16-bit kernels' byte: bits 0-3 H differs from diagonal, E, F, E2;
    bits 4-7 E, F, E2, F2 leaving the cell extend (beat opening strictly)."""
    p = pins.normalise(p)
    H, E, F, E2, F2, hds = V[(t, q)]
    b = (H != hds) | ((H != E) << 1) | ((H != F) << 2) | ((H != E2) << 3)
    hoe, hoe2 = H - p['q'] - p['e'], H - p['q2'] - p['e2']
    if E - p['e'] > hoe: b |= 16
    if F - p['e'] > hoe: b |= 32
    if E2 - p['e2'] > hoe2: b |= 64
    if F2 - p['e2'] > hoe2: b |= 128
    return b

def kernel_byte(V, t, q, p):
    """The int32 kernel's byte: bits 0-2 the index of H's source (first equal
    of diagonal, E, F, E2, F2); bits 3-6 E, F, E2, F2 leaving the cell extend."""
    p = pins.normalise(p)
    H, E, F, E2, F2, hds = V[(t, q)]
    src = 0 if H == hds else 1 if H == E else 2 if H == F else 3 if H == E2 else 4
    hoe, hoe2 = H - p['q'] - p['e'], H - p['q2'] - p['e2']
    b = src
    if E - p['e'] > hoe: b |= 8
    if F - p['e'] > hoe: b |= 16
    if E2 - p['e2'] > hoe2: b |= 32
    if F2 - p['e2'] > hoe2: b |= 64
    return b

def emulate(T, Q, p, C, et, eq, packed=False):
    """Fill a pair's table in the kernel's layout (C slots per lane), walk back
    from (et, eq) through 32-row windows as tb_walk does, asserting every
    index against its buffer; returns the CIGAR text and the window loads."""
    tl, ql = len(T), len(Q)
    w = p['w']
    if w < 0 or w > max(tl, ql): w = max(tl, ql)
    assert w <= 32 * C - 1
    ROW = 32 * C
    P = C // 2
    WA = 48 if (packed and C > 16) else 16
    WB = 144 if (packed and C > 16) else 80
    frame = (lambda r: (r - w) >> 1) if packed else (lambda r: ceil_div2(r - w))
    def byte_of(j):
        if not packed: return j
        lb = (j // C) * C; jl = j - lb
        return lb + (2 * jl if jl < P else 2 * (jl - P) + 1)
    r_end = et + eq
    V = dp_values(T, Q, p, w)
    table = np.full((r_end + 1) * ROW, 0xEE if not packed else 0x00, np.uint8)
    real = np.zeros((r_end + 1) * ROW, bool)
    for r in range(r_end + 1):
        B = frame(r)
        for j in range(ROW):
            t = B + j; q = r - t
            if 0 <= t < tl and 0 <= q < ql and abs(t - q) <= w:
                assert j <= w
                pos = r * ROW + byte_of(j)
                table[pos] = kernel_byte16(V, t, q, p) if packed else kernel_byte(V, t, q, p)
                real[pos] = True
    # windowed walk, as tb_walk
    runs = []
    def push(op, l):
        if runs and runs[-1][0] == op: runs[-1][1] += l
        else: runs.append([op, l])
    t, q = et, eq
    st = 5
    done = t < 0 or q < 0
    loads = 0
    while not done:
        r0 = t + q
        jc = t - frame(r0)
        ws = jc - 31
        ws = 0 if ws < 0 else (ws // WA) * WA
        ws = min(ws, ROW - WB)
        assert ws >= 0 and ws % 16 == 0 and (not packed or ws % C == 0)
        win = {}
        for lane in range(32):
            rk = r0 - lane
            if rk >= 0:
                lo = rk * ROW + ws
                assert lo >= 0 and lo + WB <= (r_end + 1) * ROW, (lo, r_end, ROW)
                win[lane] = (table[lo:lo + WB], real[lo:lo + WB])
        loads += 1
        while True:
            if t < 0 or q < 0:
                if t < 0 and q >= 0: push('I', q + 1)
                if q < 0 and t >= 0: push('D', t + 1)
                done = True
                break
            r = t + q
            if r < r0 - 31: break
            j = byte_of(t - frame(r)) - ws
            assert 0 <= j < WB, (j, t, q, r0, ws)
            b = int(win[r0 - r][0][j])
            assert win[r0 - r][1][j], "read a slot that is not a band cell"
            if st > 5:
                k = st - 5
                bit = (1 << (3 + k)) if packed else (1 << (2 + k))
                st = k if (b & bit) else 5
            if st == 5:
                if packed:
                    nz = (~b) & 0xf
                    st = (nz & -nz).bit_length() - 1 if nz else 4
                else:
                    st = b & 7
                assert st <= 4
            if st == 0:
                push('M', 1); t -= 1; q -= 1; st = 5
            elif st & 1:
                push('D', 1); t -= 1; st += 5
            else:
                push('I', 1); q -= 1; st += 5
    runs.reverse()
    return "".join(f"{l}{op}" for op, l in runs), loads



PSETS = [dict(a=2, b=4, q=4, e=2, q2=24, e2=1, zdrop=400, end_bonus=0),
         dict(a=1, b=2, q=2, e=1, q2=32, e2=0, zdrop=100, end_bonus=5),
         dict(a=5, b=30, q=40, e=3, q2=80, e2=1, zdrop=200, end_bonus=0),
         dict(a=2, b=1, q=0, e=1, q2=3, e2=0, zdrop=-1, end_bonus=0)]


@pytest.mark.parametrize("C", [4, 8, 16, 24])
@pytest.mark.parametrize("packed", [False, True])
def test_walk_reads_only_band_cells_and_returns_the_oracle_cigar(C, packed):
    rng = np.random.default_rng(5 + C + 100 * packed)
    done = 0
    for it in range(10):
        p = dict(PSETS[it % len(PSETS)])
        p["w"] = int(rng.integers(1, 32 * C))
        n = int(rng.integers(1, 160))
        T = rng.integers(0, 4, n).astype(np.uint8)
        Q = []
        for b in T:
            u = rng.random()
            if u < 0.06:
                Q.append((b + 1) % 4)
            elif u < 0.1:
                continue
            elif u < 0.14:
                Q.extend([b, int(rng.integers(0, 4))])
            else:
                Q.append(b)
        Q = np.array(Q or [0], np.uint8)
        sc = tuple(p[k] for k in ("a", "b", "q", "e", "q2", "e2", "w", "zdrop", "end_bonus"))
        r = O.align_pair(T, Q, sc)
        et, eq = O.end_cell(r, len(Q))
        if et < 0 or eq < 0:
            continue
        ops, _ = O.traceback_pair(T, Q, sc, et, eq)
        got, _ = emulate(T, Q, p, C, et, eq, packed)
        assert got == O.cigar_string(ops)
        done += 1
    assert done >= 5
