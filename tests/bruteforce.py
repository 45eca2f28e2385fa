"""Independent brute-force checks used to pin the oracle.

These helpers restate the paper's definitions on plain coordinates (no
Morton arithmetic, no shared code with the oracle or the CUDA library) so
that a slip in either implementation shows up as a disagreement:

* mode_pyramid: Sec. 3.1 / 3.4 -- each coarser node takes the most frequent
  of its 8 children, ties to the first occurrence in the child array.
* expected_ops: Sec. 3.2 / Alg. 2 -- for every coded child, the list of
  operations that would reproduce its label, evaluated independently, so a
  test can check that the emitted one is the first applicable in the order
  R_p, R_x, R_y, R_z, P_0, P_delta, P_a.
"""
import numpy as np

CHILD = [(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]  # (dx, dy, dz) of child index c


def mode_pyramid(brick):
    """Levels 0..N as arrays indexed [z, y, x], plus 'constant subtree' flags."""
    b = brick.shape[0]
    N = b.bit_length() - 1
    labs = [brick.astype(np.uint64)]
    csts = [np.ones_like(brick, dtype=bool)]
    for l in range(1, N + 1):
        B = b >> l
        prev, pc = labs[-1], csts[-1]
        lab = np.zeros((B, B, B), np.uint64)
        cst = np.zeros((B, B, B), bool)
        for z in range(B):
            for y in range(B):
                for x in range(B):
                    kids = [prev[2 * z + dz, 2 * y + dy, 2 * x + dx] for (dx, dy, dz) in CHILD]
                    counts = {}
                    for k in kids:
                        counts[k] = counts.get(k, 0) + 1
                    top = max(counts.values())
                    lab[z, y, x] = next(k for k in kids if counts[k] == top)
                    cst[z, y, x] = top == 8 and all(pc[2 * z + dz, 2 * y + dy, 2 * x + dx] for (dx, dy, dz) in CHILD)
        labs.append(lab)
        csts.append(cst)
    return labs, csts


def morton_order(B):
    """Coordinates (x, y, z) of a B^3 grid sorted by interleaved bits, x lowest."""
    def key(p):
        x, y, z = p
        k = 0
        for bit in range(B.bit_length()):
            k |= ((x >> bit) & 1) << (3 * bit)
            k |= ((y >> bit) & 1) << (3 * bit + 1)
            k |= ((z >> bit) & 1) << (3 * bit + 2)
        return k
    pts = [(x, y, z) for z in range(B) for y in range(B) for x in range(B)]
    return sorted(pts, key=key)


def coded_children(brick):
    """Children in stream order, as (level of child, (x,y,z) of child, parent label, child label, stop)."""
    labs, csts = mode_pyramid(brick)
    N = len(labs) - 1
    out = []
    for l in range(N, 0, -1):
        B = brick.shape[0] >> l
        for (px, py, pz) in morton_order(B):
            if csts[l][pz, py, px]:
                continue
            for (dx, dy, dz) in CHILD:
                q = (2 * px + dx, 2 * py + dy, 2 * pz + dz)
                v = labs[l - 1][q[2], q[1], q[0]]
                stop = bool(csts[l - 1][q[2], q[1], q[0]]) if l - 1 >= 1 else False
                out.append((l - 1, q, labs[l][pz, py, px], v, stop))
    return out, labs


def neighbour(labs, lc, q, axis):
    """Label that neighbour reuse along `axis` gives child q on level lc, or None if outside the brick.

    Even coordinate along the axis: the node one step back on the same level.
    Odd coordinate: the node one step forward is not decoded yet, so its parent.
    """
    B = labs[lc].shape[0]
    n = list(q)
    if q[axis] % 2 == 0:
        n[axis] -= 1
        if n[axis] < 0:
            return None
        return labs[lc][n[2], n[1], n[0]]
    n[axis] += 1
    if n[axis] >= B:
        return None
    return labs[lc + 1][n[2] // 2, n[1] // 2, n[0] // 2]


def check_first_applicable(brick, palette, int_nib, leaf_nib):
    """Walk the streams next to an independent evaluation; returns a list of problems (empty = ok)."""
    kids, labs = coded_children(brick)
    streams = {"int": list(int(v) for v in int_nib), "leaf": list(int(v) for v in leaf_nib)}
    pos = {"int": 0, "leaf": 0}
    pal = [palette[0]]
    ip = 0
    problems = []
    for (lc, q, parent, v, stop) in kids:
        s = "int" if lc >= 1 else "leaf"
        nib = streams[s][pos[s]]
        pos[s] += 1
        op, sbit = nib & 7, nib >> 3
        if sbit != int(stop):
            problems.append(("stop", lc, q, sbit, stop))
        applicable = []
        if v == parent:
            applicable.append(0)
        for a in range(3):
            nv = neighbour(labs, lc, q, a)
            if nv is not None and nv == v:
                applicable.append(1 + a)
        if pal[ip] == v:
            applicable.append(4)
        back = [d for d in range(16) if ip - 1 - d >= 0 and pal[ip - 1 - d] == v]
        if back:
            applicable.append(5)
        applicable.append(6)
        if op != applicable[0]:
            problems.append(("op", lc, q, op, applicable))
        if op == 5:
            d = streams[s][pos[s]]
            pos[s] += 1
            if d != back[0]:
                problems.append(("delta", lc, q, d, back[0]))
        if op == 6:
            pal.append(v)
            ip += 1
    if pos["int"] != len(streams["int"]) or pos["leaf"] != len(streams["leaf"]):
        problems.append(("length", pos, {k: len(x) for k, x in streams.items()}))
    if [int(x) for x in pal] != [int(x) for x in palette]:
        problems.append(("palette", pal, list(palette)))
    return problems


def voronoi_brick(rng, b, n_sites, n_labels):
    """Small Voronoi-like brick (nearest of a few random sites) with labels drawn from n_labels values."""
    sites = rng.integers(0, b, size=(n_sites, 3))
    labels = rng.integers(0, n_labels, size=n_sites).astype(np.uint32) * 7 + 3
    z, y, x = np.meshgrid(np.arange(b), np.arange(b), np.arange(b), indexing="ij")
    d = (x[..., None] - sites[:, 0]) ** 2 + (y[..., None] - sites[:, 1]) ** 2 + (z[..., None] - sites[:, 2]) ** 2
    return labels[np.argmin(d, axis=-1)].astype(np.uint32)


def read_golden(path):
    rec = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, _, v = line.partition(":")
            rec[k.strip()] = [int(t) for t in v.split()]
    b = rec["b"][0]
    brick = np.array(rec["brick"], np.uint32).reshape(b, b, b)
    return brick, rec["palette"], rec["interior"], rec["leaf"]
