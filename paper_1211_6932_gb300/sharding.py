"""Assignment of independent instances to ranks (the batch is embarrassingly parallel:
instances never exchange data, so each rank advances its own share and no collective
touches the data path)."""


def shard(weights, world, rank):
    """Indices of the instances rank `rank` of `world` owns: contiguous runs in the given
    order, cut where the running total of `weights` (e.g. node counts) crosses
    k / world of the sum, so shares differ by at most one instance's weight.  Every index
    belongs to exactly one rank; deterministic."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d out of range for world %d" % (rank, world))
    total = float(sum(weights))
    lo_cut, hi_cut = total * rank / world, total * (rank + 1) / world
    out, run = [], 0.0
    for i, w in enumerate(weights):
        mid = run + 0.5 * w  # an instance goes to the rank whose interval holds its middle
        if lo_cut <= mid < hi_cut or (rank == world - 1 and mid >= hi_cut):
            out.append(i)
        run += w
    return out
