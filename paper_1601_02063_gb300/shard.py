"""Work partition across ranks (one process per GPU).

Rays are independent (Section 1: no communication between the per-pixel threads), so
several GPUs either render images of their own (weak scaling) or split one image into
contiguous row slabs (strong scaling), each rank writing its own slab; neither needs a
collective on the data path.  The only exchange is the timing aggregate of a benchmark:
the slowest rank's time and the sum of the ranks' Runge-Kutta attempts and rays.
"""
from __future__ import annotations


def row_range(n_beta: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [j0, j1) of rank `rank` of `world`: contiguous slabs whose sizes differ by at
    most one row, the first n_beta % world ranks taking the larger ones."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(n_beta), world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def row_shard(scene: dict, rank: int, world: int) -> dict | None:
    """The rank's rows of `scene` as a scene of their own (None if the rank has no row).
    The window is cut at row boundaries, so the shard's pixel centres are those of the
    full image: beta_j = beta_min + (j + 1/2) dbeta with the full image's dbeta."""
    j0, j1 = row_range(scene["n_beta"], rank, world)
    if j1 <= j0:
        return None
    db = (scene["beta_max"] - scene["beta_min"]) / scene["n_beta"]
    return dict(scene, beta_min=scene["beta_min"] + j0 * db, beta_max=scene["beta_min"] + j1 * db,
                n_beta=j1 - j0)


def aggregate(total_ms: float, steps: float, rays: float, dist=None):
    """(slowest rank's time, sum of attempts, sum of rays) over the process group (or this
    process alone when `dist` is None or not initialised).  CPU tensors: works on gloo."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(total_ms), float(steps), float(rays)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64)
    s = torch.tensor([float(steps), float(rays)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t[0]), float(s[0]), float(s[1])
