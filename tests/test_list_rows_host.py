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
left unwritten back slots in kept rows near the capacity.  The warp-per-
particle build of small systems stores each accepted entry at the slot the
per-thread build's shift queue gives it; the last test checks that the two
write the same row, entry for entry."""
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


def _thread_row(entries, cap, sentinel):
    """Row contents of the per-thread build: (j, image) entries in candidate
    order; a 4-register shift queue (newest first) stored as one chunk when
    four front entries are complete, image entries from the back."""
    row = np.full(cap, -1, np.int64)
    q = [0, 0, 0, 0]
    nf = nb = 0
    for j, img in entries:
        if not img:
            q = [j] + q[:3]
            nf += 1
            if nf % 4 == 0 and nf + nb <= cap:
                row[nf - 4:nf] = q
        else:
            if nb < cap:
                row[cap - 1 - nb] = j
            nb += 1
    kept = (nf + 3) // 4 * 4 + nb <= cap
    if kept and nf % 4:
        for _ in range(nf % 4, 4):
            q = [sentinel] + q[:3]
        row[nf // 4 * 4:nf // 4 * 4 + 4] = q
    return row, kept


def _warp_row(cands, cap, sentinel):
    """Row contents of the warp-per-particle build: candidates in blocks of
    32 lanes; a ballot per block, each accepted lane storing at
    nf + (accepted lanes below it), the front slot reversed within its chunk
    of four; sentinels from lanes nf % 4 .. 3 at the end."""
    row = np.full(cap, -1, np.int64)
    nf = nb = 0
    for b0 in range(0, len(cands), 32):
        blk = cands[b0:b0 + 32]
        for img in (False, True):
            acc = [j for j, inside, im in blk if inside and im == img]
            for k, j in enumerate(acc):
                if not img:
                    e = nf + k
                    pos = (e & ~3) + 3 - (e & 3)
                    if pos < cap:
                        row[pos] = j
                else:
                    if nb + k < cap:
                        row[cap - 1 - (nb + k)] = j
            if img:
                nb += len(acc)
            else:
                nf += len(acc)
    kept = (nf + 3) // 4 * 4 + nb <= cap
    if kept:
        for lane in range(nf & 3, 4 if nf & 3 else 0):
            row[(nf & ~3) + 3 - lane] = sentinel
    return row, kept


def test_warp_and_thread_builds_write_identical_rows():
    """The slot rule of the warp build reproduces the per-thread build's
    rows, entry for entry, in every kept row (runs carry one image code, so
    a block of 32 candidates holds front or image entries, never both)."""
    rng = np.random.default_rng(3)
    for _ in range(3000):
        cap = 4 * int(rng.integers(1, 40))
        cands = []
        j = 0
        for _ in range(int(rng.integers(1, 8))):  # runs
            img = bool(rng.random() < 0.3)
            m = int(rng.integers(0, 90))
            p = rng.uniform(0.05, 0.9)
            # a run is tested in blocks of 32 from its own start
            run = [(j + t, bool(rng.random() < p), img) for t in range(m)]
            j += m
            for b0 in range(0, m, 32):
                blk = run[b0:b0 + 32]
                cands.append(blk)
        sentinel = j + 1
        thread_entries = [(jj, im) for blk in cands for jj, inside, im in blk if inside]
        rt, kt = _thread_row(thread_entries, cap, sentinel)
        # the warp build, block by block (each block is padded to 32 lanes)
        flat = []
        for blk in cands:
            flat.extend(blk + [(-1, False, blk[0][2])] * (32 - len(blk)))
        rw, kw = _warp_row(flat, cap, sentinel)
        assert kt == kw
        if kt:
            assert (rt == rw).all(), (cap, rt, rw)
