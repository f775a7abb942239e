"""Host model of the shared-tap weight-gradient kernel's tile schedule.

The kernel (csrc/unet.cu, wgrad_tap_kernel) keeps the dZ rows of a run of
row tiles in a ring of R = S + 2 slots plus two mirror slots (R, R + 1 repeat
slots 0, 1), so that the three rows a tile reads are always evenly spaced:

  * a CTA takes tiles t in [ntiles q / per, ntiles (q + 1) / per) in (image,
    strip, row) order; a tile whose row is 0, or the first of the run, starts
    a fresh window at slot 0 (rows y - 1, y, y + 1 into slots 0, 1, 2 and
    rows y - 1, y again into slots R, R + 1); any other tile moves the window
    down one slot and loads row y + 1 into slot (ws + 2) mod R (and into its
    mirror when that slot is 0 or 1);
  * before tile j's copies, its producer waits for every tile up to
    max(run - 1, j - S) to have been read by the tensor cores, where run is
    the tile that started the current window run.

This model replays those rules on the host and checks the two properties
the kernel relies on: every window reads the rows y - 1, y, y + 1 of its own
image and strip, and no copy overwrites a slot whose previous rows some tile
past the waited-for one still reads.  Several producers issue the tiles of a
CTA out of order, so the wait must cover the previous run (the rule without
it is shown to fail below).
"""
import pytest


def _replay(H, segs, B, per, S, with_run_wait=True):
    """Returns None if the schedule is safe, else a description of the first
    violation."""
    R = S + 2
    ntiles = B * segs * H
    for q in range(per):
        tb, te = ntiles * q // per, ntiles * (q + 1) // per
        content = {}   # slot -> (image, strip, row)
        readers = {}   # slot -> tiles that read its current content
        ws = 0
        run = 0
        for j in range(te - tb):
            t = tb + j
            strip_all = t // H
            y = t - strip_all * H
            b, strip = strip_all // segs, strip_all % segs
            fresh = j == 0 or y == 0
            ws = 0 if fresh else (0 if ws + 1 == R else ws + 1)
            if fresh:
                run = j
            if with_run_wait:
                upto = max(run - 1, j - S)
            else:
                upto = j - 1 if fresh else j - S
            if fresh:
                writes = [(0, y - 1), (1, y), (2, y + 1), (R, y - 1), (R + 1, y)]
            else:
                sn = ws + 2 if ws + 2 < R else ws + 2 - R
                writes = [(sn, y + 1)] + ([(R + sn, y + 1)] if sn < 2 else [])
            for slot, row in writes:
                for r in readers.get(slot, []):
                    if r > upto:
                        return f"CTA {q} tile {j}: slot {slot} still read by tile {r} (waited up to {upto})"
                readers[slot] = []
                content[slot] = (b, strip, row)
            for k in range(3):
                slot = ws + k
                assert slot <= R + 1, "window past the mirror slots"
                want = (b, strip, y - 1 + k)
                if content.get(slot) != want:
                    return f"CTA {q} tile {j}: slot {slot} holds {content.get(slot)}, wants {want}"
                readers.setdefault(slot, []).append(j)
    return None


# (rows, strips, images, CTAs per slice/chunk pair, stages): the 2048x1024
# level-0 launch, the test networks' levels, and short strips that make runs
# cross strips and images and wrap the ring many times
CASES = [(1024, 16, 1, 152, 8), (512, 8, 1, 152, 8), (256, 4, 1, 3, 8), (8, 4, 1, 3, 8),
         (24, 4, 2, 3, 8), (24, 4, 2, 1, 8), (40, 2, 1, 1, 8), (6, 2, 1, 3, 8), (2, 4, 2, 5, 8),
         (7, 1, 1, 1, 5), (13, 3, 2, 2, 6)]


@pytest.mark.parametrize("H,segs,B,per,S", CASES)
def test_ring_schedule_reads_the_right_rows_and_never_overwrites_a_live_slot(H, segs, B, per, S):
    assert _replay(H, segs, B, per, S) is None


def test_mirror_slots_are_used():
    # runs long enough to wrap the ring do read the mirror slots (R, R + 1)
    R = 8 + 2
    H, segs, B, per, S = 40, 2, 1, 1, 8
    ntiles = B * segs * H
    ws, uses = 0, 0
    for j in range(ntiles):
        y = j % H
        ws = 0 if (j == 0 or y == 0) else (0 if ws + 1 == R else ws + 1)
        uses += sum(1 for k in range(3) if ws + k >= R)
    assert uses > 0


def test_waiting_only_for_tile_j_minus_s_is_not_enough_after_a_new_strip():
    # without the wait for the previous run, a tile just after a strip change
    # may overwrite a slot that a tile of the previous strip still reads
    assert _replay(8, 4, 1, 3, 8, with_run_wait=False) is not None
