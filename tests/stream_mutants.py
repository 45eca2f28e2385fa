"""Edits of a brick's op streams for the malformed- and unusual-stream tests (test infrastructure).

A stream is the oracle's nibble sequence of one brick (Sec. 3.2 / 3.3): op nibbles (op | stop << 3) in stream
order, each P_delta (op 5) followed by its delta nibble.  The edits keep that grammar unless they are meant to
break it: an op replaced by another reuse op, by P_0, P_delta (a delta nibble inserted) or P_a; a P_delta's
delta changed or removed with the op; op 7; a stop bit set on a leaf or flipped on an interior op.  Whether an
edited stream is valid is for the decoders to decide; the tests compare the CUDA decoder's verdict and labels
with the oracle's.
"""
import numpy as np

OP_P0, OP_PD, OP_PA = 4, 5, 6


def parse(stream):
    """nibbles -> list of [op nibble, delta or None]"""
    ops, i, s = [], 0, [int(x) for x in stream]
    while i < len(s):
        o = s[i]
        if (o & 7) == OP_PD and i + 1 < len(s):
            ops.append([o, s[i + 1]])
            i += 2
        else:
            ops.append([o, None])
            i += 1
    return ops


def flatten(ops):
    out = []
    for o, d in ops:
        out.append(o)
        if d is not None:
            out.append(d)
    return np.asarray(out, np.uint8)


def mutate_one(rng, ops, leaf):
    """One random edit of an op list in place."""
    k = int(rng.integers(len(ops)))
    o, d = ops[k]
    stop, op = o & 8, o & 7
    kind = int(rng.integers(9))
    if kind <= 1:  # another reuse op or P_0
        new = int(rng.choice([x for x in (0, 1, 2, 3, OP_P0) if x != op]))
        ops[k] = [new | stop, None]
    elif kind == 2:  # P_delta with a small delta
        ops[k] = [OP_PD | stop, int(rng.integers(0, 4))]
    elif kind == 3:  # any delta
        ops[k] = [OP_PD | stop, int(rng.integers(0, 16))]
    elif kind == 4:  # P_a
        ops[k] = [OP_PA | stop, None]
    elif kind == 5:  # a palette op back to P_0 (drops a P_a or a delta)
        ops[k] = [OP_P0 | stop, None] if op in (OP_PD, OP_PA) else [(op ^ 1) | stop if op < 4 else OP_P0 | stop, None]
    elif kind == 6:  # op 7
        ops[k] = [7 | stop, None]
    elif kind == 7:  # stop bit: set on a leaf, flipped on an interior op
        ops[k] = [o | 8 if leaf else o ^ 8, d]
    else:  # two ops exchanged
        j = int(rng.integers(len(ops)))
        ops[k], ops[j] = ops[j], ops[k]


def mutants(rng, ni, nl, count, max_edits=3, leaf_share=0.7):
    """`count` edited (interior, leaf) stream pairs of one brick."""
    out = []
    for _ in range(count):
        oi, ol = parse(ni), parse(nl)
        for _ in range(int(rng.integers(1, max_edits + 1))):
            if ol and (rng.random() < leaf_share or not oi):
                mutate_one(rng, ol, True)
            elif oi:
                mutate_one(rng, oi, False)
        out.append((flatten(oi), flatten(ol)))
    return out
