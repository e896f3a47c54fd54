"""Host replicas of two pieces of the FP32 pair kernel's index arithmetic, checked for
every size they can meet (no GPU): the shared-memory ring split by plane group, and the
column wrap of full-width strips.  The kernel's own results are checked against the
oracle by the GPU parity tests; these make sure the schedules are right for chunk
lengths and widths the GPU tests do not enumerate.

Ring: rows of a sweep are issued in order; row j's three groups of planes ("ahead",
"centre", "behind") go to rings of 3, 4 and 5 slots; row j is issued right after the row
barrier of step j - 3 (rows 0..3 before the loop; row 0 without its ahead planes) and
waited for at step j - 1; step s reads the ahead planes of row s+1, the centre planes of
row s, the behind planes of row s-1, and at a wall row the ahead and behind planes of row
s itself (bounce-back).  Five row barriers are reused round robin.

Full width: a CTA of NT threads covers an instance of nx <= 2 NT columns; thread t owns
columns 2t and 2t+1 and reads the left neighbour of its first column and the right
neighbours of both, wrapped across the row."""
import pytest

DA, DC, DB, NB, LEAD = 3, 4, 5, 5, 3


def ring_schedule_ok(nload):
    slot = {"A": [None] * DA, "C": [None] * DC, "B": [None] * DB}
    bar = [None] * NB
    issued, waited = [], [0]

    def issue(j):
        if bar[j % NB] is not None:
            assert bar[j % NB] < waited[0], ("barrier reused before its row was waited", j)
        bar[j % NB] = j
        if j >= 1:
            slot["A"][j % DA] = j
        slot["C"][j % DC] = j
        slot["B"][j % DB] = j
        issued.append(j)

    def read(group, sl, row):
        assert slot[group][sl] == row, (nload, group, sl, slot[group][sl], row)
        assert row < waited[0]

    for j in range(min(nload, LEAD + 1)):
        issue(j)
    sa, sc, sb = 2 % DA, 1 % DC, 0
    for s in range(1, nload - 1):
        while waited[0] <= s + 1:
            assert waited[0] in issued
            waited[0] += 1
        read("A", sa, s + 1)
        read("C", sc, s)
        read("B", sb, s - 1)
        read("A", s % DA, s)  # bounce-back at a wall row
        read("B", s % DB, s)
        if s + LEAD < nload:  # after the row barrier of step s
            issue(s + LEAD)
        sa, sc, sb = (sa + 1) % DA, (sc + 1) % DC, (sb + 1) % DB
    return True


@pytest.mark.parametrize("nload", range(5, 204))
def test_plane_group_ring_schedule(nload):
    """Chunks of 1 to 200 rows (a chunk of r rows loads r + 4)."""
    assert ring_schedule_ok(nload)


def test_plane_group_ring_rejects_a_shorter_ring():
    """The check has teeth: with an ahead ring of 2 slots a read finds the wrong row."""
    global DA
    keep = DA
    try:
        DA = 2
        with pytest.raises(AssertionError):
            ring_schedule_ok(40)
    finally:
        DA = keep


@pytest.mark.parametrize("nt", [32, 64, 96, 128])
def test_full_width_wrap(nt):
    seg_halo, seg, psw = 4, 2 * nt + 4, 2 * nt + 4
    for nx in range(1, 2 * nt + 1):
        loaded = (nx + 3) & ~3
        assert seg_halo + loaded <= seg
        for t in range(nt):
            c0 = 2 * t
            c_l = c0 - 1 + (nx if c0 == 0 else 0)
            c_r1 = c0 + 1 - (nx if c0 + 1 >= nx else 0)
            c_r2 = c0 + 2 - (nx if c0 + 2 >= nx else 0)
            for c in (c0, c0 + 1, c_l, c_r1, c_r2):  # every thread's reads stay in its rows
                assert 0 <= seg_halo + c < seg and 2 + c < psw
            if c0 < nx:  # owners read the right columns, inside the loaded part
                assert c_l == (c0 - 1) % nx and c_r1 == (c0 + 1) % nx
                assert max(c0, c_l, c_r1) < loaded
                if c0 + 1 < nx:
                    assert c_r2 == (c0 + 2) % nx and c_r2 < loaded
