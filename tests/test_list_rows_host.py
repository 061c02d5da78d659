"""The write protocol of a Verlet-list row, modelled on the host (the
particle, batched and window list builds follow it): entries without an
image fill the row from the front in chunks (4 entries of 32 bits, or 8 of
16 bits in a window half row), written when a chunk completes and while
the front and back counts leave room; image entries fill it from the back;
at the end a row whose length (front rounded up to a chunk, plus back) fits
the capacity is kept, its last chunk padded, and any other row discarded.
The rule for an image entry is that it stays inside the row.  Checked here
over random sequences: in a kept row every counted slot was written exactly
once and front and back never overlap, and no write leaves the row.  The
former rule (write an image entry only while a whole free chunk remained)
left unwritten back slots in kept rows near the capacity."""
import numpy as np


def _roundup(k, c):
    return (k + c - 1) // c * c


def _build_row(seq, cap, chunk, back_ok):
    """seq: True for an entry without an image, False for an image entry.
    Returns (writes per slot, nf, nb, kept)."""
    writes = np.zeros(cap, np.int64)
    nf = nb = 0
    for front in seq:
        if front:
            nf += 1
            if nf % chunk == 0 and nf + nb <= cap:
                assert 0 <= nf - chunk and nf <= cap
                writes[nf - chunk:nf] += 1
        else:
            if back_ok(nf, nb, cap, chunk):
                assert 0 <= cap - 1 - nb < cap
                writes[cap - 1 - nb] += 1
            nb += 1
    need = _roundup(nf, chunk) + nb
    kept = need <= cap
    if kept and nf % chunk:
        last = (nf // chunk) * chunk
        writes[last:last + chunk] += 1  # the padded last chunk
    return writes, nf, nb, kept


def _fixed(nf, nb, cap, chunk):
    return nb < cap


def _former(nf, nb, cap, chunk):
    return _roundup(nf + 1, chunk) + nb < cap


def _check(rule, trials=20000, seed=0):
    rng = np.random.default_rng(seed)
    bad = 0
    for _ in range(trials):
        chunk = int(rng.choice([4, 8]))
        cap = chunk * int(rng.integers(2, 12))
        n = int(rng.integers(0, cap + 8))
        seq = rng.random(n) < rng.uniform(0.3, 1.0)
        writes, nf, nb, kept = _build_row(seq, cap, chunk, rule)
        if not kept:
            continue
        front = writes[:_roundup(nf, chunk)]
        back = writes[cap - nb:] if nb else writes[:0]
        ok = (front == 1).all() and (back == 1).all() and _roundup(nf, chunk) <= cap - nb
        bad += not ok
    return bad


def test_kept_rows_are_fully_written_with_the_image_entries_inside_the_row():
    assert _check(_fixed) == 0


def test_the_former_rule_left_unwritten_image_slots():
    assert _check(_former) > 0
    # the smallest case: a 4-entry chunk, capacity 8, four front entries then
    # four image entries; the row fits (4 + 4 = 8) but the former rule wrote
    # none of the four image entries
    writes, nf, nb, kept = _build_row([True] * 4 + [False] * 4, 8, 4, _former)
    assert kept and nf == 4 and nb == 4 and (writes[4:] == 0).all()
    writes, nf, nb, kept = _build_row([True] * 4 + [False] * 4, 8, 4, _fixed)
    assert kept and (writes == 1).all()
