"""Oracle, grouping side: scenes, frame tuples / groups, and the Figure 1 frame-store layout.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Pure integer logic.

Section 3.3 ("Internal Design"): frames are always grouped within a scene;
an interpolation network gets the scene's last frame duplicated; a last group
short of frames recycles frames of the previous group; a scene shorter than
the network's input count duplicates its last frame further.  Scene changes
arrive as a per-frame property (Section 3.2, "End User Usage").  Readings:

* a flag on frame k means frame k starts a new scene (cut between k-1 and k);
  the clip's first and last frames bound scenes too;
* sliding window of T = 2r+1 frames, one output per input frame t:
  j_k = clamp(t - r + k, s0(t), s1(t)), k = 0..T-1 (edge frames replicated,
  never mixed across a cut);
* group model with n consumed frames per run (Section 3.1 flags): with the
  Extra-frame flag a run takes n+1 frames; runs tile the scene by n; indices
  past the scene end take the scene's last frame (interpolation: the last frame
  duplicated; short scene: further duplication); a short last group of a
  non-interpolating network is shifted back to end at the scene end
  (recycling earlier frames) as long as the scene is long enough.
"""
from __future__ import annotations


def scenes_from_flags(flags, nframes: int):
    """List of (s0, s1) inclusive scene bounds; flags[k] true = frame k starts a scene."""
    starts = [0] + [k for k in range(1, nframes) if flags[k]]
    ends = [s - 1 for s in starts[1:]] + [nframes - 1]
    return list(zip(starts, ends))


def scene_of(t: int, scenes):
    for s0, s1 in scenes:
        if s0 <= t <= s1:
            return s0, s1
    raise IndexError(t)


def tuple_indices(t: int, T: int, s0: int, s1: int):
    """Source frame indices of output t's tuple (sliding window, edge replication)."""
    r = (T - 1) // 2
    return [min(max(t - r + k, s0), s1) for k in range(T)]


def tuple_map(flags, nframes: int, T: int):
    """Per output frame t (one per input frame): its T source indices."""
    scenes = scenes_from_flags(flags, nframes)
    return [tuple_indices(t, T, *scene_of(t, scenes)) for t in range(nframes)]


def group_runs(s0: int, s1: int, n: int, extra: bool, interp: bool):
    """Network runs covering one scene [s0, s1] under the group model.

    Returns a list of (inputs, skip): the run's input frame indices and how
    many of its leading frames were already covered by an earlier run.
    Runs nominally start at s0, s0+n, ...; each takes n (+1 with Extra frame)
    frames; indices past s1 take s1 (duplication of the scene's last frame).
    A non-interpolating network's last run that would pass s1 is moved back to
    end at s1 when the scene holds enough frames (recycling frames of the
    previous group); ``skip`` then counts the recycled frames.
    """
    need = n + (1 if extra else 0)
    length = s1 - s0 + 1
    runs = []
    for nominal in range(s0, s1 + 1, n):
        start = nominal
        if not interp and start + need - 1 > s1 and length >= need:
            start = s1 - need + 1
        runs.append(([min(start + k, s1) for k in range(need)], nominal - start))
    return runs


def group_output_count(n: int, interp: bool, double: bool) -> int:
    """Frames emitted per run: 2n with Double frame, else n (Section 3.1 flags)."""
    return 2 * n if double else n


def fig1_layout(n: int, b: int):
    """Frame-store layout for a batch of b groups of n+1 frames (Section 3.3, Figure 1).

    The store has b rows and n+1 columns and is addressed column first
    (address = column * b + row).  Column 0 only uses its last row, holding
    the batch's first frame; the other b-1 cells of column 0 are unused.
    Column 1 holds the groups' last frames ((r+1) n for row r); column k+1
    (k = 1..n-1) holds frame r*n + k.  Input slot k of the network (the k-th
    frame of every group) is then b contiguous cells: slot 0 starts at address
    b-1, slot n at address b, slot k (1 <= k < n) at address (k+1) b.  The
    batch uses b n + 1 cells.

    Returns (grid, slot_start) where grid[row][col] is the frame index
    relative to the batch's first frame (None = unused) and slot_start[k] is
    the address of slot k's first cell.
    """
    grid = [[None] * (n + 1) for _ in range(b)]
    grid[b - 1][0] = 0
    for r in range(b):
        grid[r][1] = (r + 1) * n
        for k in range(1, n):
            grid[r][k + 1] = r * n + k
    slot_start = [b - 1] + [(k + 1) * b for k in range(1, n)] + [b]
    return grid, slot_start


def fig1_slot_frames(grid, slot_start, n: int, b: int):
    """Read each input slot's b frames back out of the column-first store."""
    flat = [grid[a % b][a // b] for a in range(b * (n + 1))]
    return [flat[slot_start[k]:slot_start[k] + b] for k in range(n + 1)]


def fig1_next_batch_copy(n: int, b: int, rolling: bool = True):
    """(src_address, dst_address) of the single copy that prepares the next batch.

    The next batch's first frame is this batch's last frame (b n), stored at
    column 1, row b-1 (address 2b - 1).  In the figure's rolling store the
    next batch's block begins one cell before this batch's end, so that frame
    is copied onto the last cell of this batch (address (n+1) b - 1, which
    holds frame (b-1) n + n - 1: "6 to 5" for n = 3, b = 2).  A store reused in
    place copies it to column 0, row b-1 (address b - 1) instead.
    """
    src = 2 * b - 1
    return (src, (n + 1) * b - 1) if rolling else (src, b - 1)
