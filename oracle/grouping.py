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
  Extra-frame flag a run takes n+1 frames, the last being the next group's
  first; runs tile the scene by n; indices past the scene end take the
  scene's last frame (the interpolation network's last frame duplicated, and
  a scene shorter than n duplicated further); a last group whose consumed
  frames pass the scene end is moved back to end there, recycling frames of
  the previous group, when the scene holds n frames;
* every consumed frame of the scene gives its outputs exactly once
  ("a complete set of rules to always output required number of frames"):
  2 per frame with Interpolation (doubled frame rate) or Double frame (2n
  network outputs per run), else 1; outputs an earlier run already emitted,
  and outputs of duplicated frames past the scene end, are not emitted;
* Interpolation without Double frame: the run's input frames are output as
  they are, each followed by the network output that is its intermediate
  frame (Section 3.1, "Double frame" flag).
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


def group_runs(s0: int, s1: int, n: int, extra: bool):
    """Network runs covering one scene [s0, s1] under the group model.

    Returns a list of (inputs, skip, count): the run's input frame indices, how
    many of its leading consumed frames an earlier run already covered, and
    how many consumed frames it covers for the first time.  Runs nominally
    start at s0, s0+n, ...; each consumes n frames and takes n (+1 with Extra
    frame) frames; indices past s1 take s1 (duplication of the scene's last
    frame).  A run whose consumed frames would pass s1 is moved back to end at
    s1 when the scene holds n frames (recycling frames of the previous group);
    ``skip`` then counts the recycled frames.  The counts of a scene add up to
    its length.
    """
    need = n + (1 if extra else 0)
    length = s1 - s0 + 1
    runs = []
    for nominal in range(s0, s1 + 1, n):
        start = nominal
        if start + n - 1 > s1 and length >= n:
            start = s1 - n + 1
        count = min(start + n - 1, s1) - nominal + 1
        runs.append(([min(start + k, s1) for k in range(need)], nominal - start, count))
    return runs


def group_output_count(n: int, interp: bool, double: bool) -> int:
    """Network outputs per run: 2n with Double frame, else n (Section 3.1 flags)."""
    return 2 * n if double else n


def outputs_per_frame(interp: bool, double: bool) -> int:
    """Output frames per consumed input frame: 2 at doubled frame rate (Interpolation,
    or Double frame's 2n outputs per n frames), else 1."""
    return 2 if (interp or double) else 1


def group_outputs(flags, nframes: int, n: int, extra: bool, interp: bool, double: bool):
    """Every output of a group-model stream, in presentation order.

    Each entry is ("net", inputs, k) -- output k of the network run on frames
    ``inputs`` -- or ("pass", i) -- input frame i output as it is.  A run's
    consumed frame j gives, with Interpolation and without Double frame, the
    frame itself then network output j (its intermediate frame); with Double
    frame, network outputs 2j and 2j+1; otherwise network output j.
    """
    q = outputs_per_frame(interp, double)
    out = []
    for s0, s1 in scenes_from_flags(flags, nframes):
        for inputs, skip, count in group_runs(s0, s1, n, extra):
            for j in range(skip, skip + count):
                if interp and not double:
                    out.append(("pass", inputs[j]))
                    out.append(("net", tuple(inputs), j))
                else:
                    out.extend(("net", tuple(inputs), q * j + e) for e in range(q))
    return out


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
