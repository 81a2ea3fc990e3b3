"""Data-parallel and streamed forms of the Accum reverse passes: one process
per GPU, the units (points of a mixture, observations of a reprojection)
sharded across ranks, parameters replicated; on each rank the points may also
stream from host memory in chunks (gmm_vjp_from_host).

Accum sums are associative (Sec. 2.3.2), so each rank accumulates over its own
shard and one all-reduce (sum) of the accumulated vector combines them; the
per-unit statistics (logsumexp per point, residual per observation) never
leave their rank. For the mixture the vector is the exchange vector of
``gmm_vjp_partial``; for the reprojection it is the pair of cotangent arrays
``(d_cams, d_pts)`` themselves.

Ranks, world size and the process group come from ``torch.distributed``;
without an initialised group (or with one rank) no collective runs.
"""
import torch

from . import _lib


def _world(group=None) -> int:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def shard_range(n: int, rank: int, world: int, align: int = 128):
    """[begin, end) of rank's contiguous share of n units, in rank order: whole
    blocks of ``align`` units (so a shard of points starts on a 128-point
    tile), the extra blocks on the last ranks so that the one partial block
    lands on a rank with one block more; shares differ by at most ``align``
    units, every unit is in exactly one share, and a rank may get none."""
    if n < 0 or world < 1 or not 0 <= rank < world or align < 1:
        raise ValueError("shard_range: need n >= 0, world >= 1, 0 <= rank < world, align >= 1")
    blocks = (n + align - 1) // align
    base, extra = divmod(blocks, world)
    first_extra = world - extra
    b0 = rank * base + max(0, rank - first_extra)
    b1 = b0 + base + (1 if rank >= first_extra else 0)
    return min(n, b0 * align), min(n, b1 * align)


def combine(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum ``t`` over all ranks in place (one all-reduce); returns ``t``."""
    if _world(group) > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def total_units(n_local: int, device, group=None) -> int:
    """Sum of the ranks' unit counts (one all-reduce of an int64)."""
    if _world(group) == 1:
        return int(n_local)
    t = torch.tensor([int(n_local)], dtype=torch.int64, device=device)
    combine(t, group)
    return int(t.item())


def gmm_vjp(x_shard, alpha, mu, q, l, gamma=1.0, m=0, prec=_lib.PREC_FP32, seed=1.0, n_total=None,
            d_alpha=None, d_mu=None, d_q=None, d_l=None, out=None, ws=None, exch=None, status=None,
            stream=None, group=None):
    """seed * grad f of the mixture over the points of every rank, added into
    (d_alpha, d_mu, d_q, d_l) on every rank; ``out`` (float64 [1], optional)
    receives f. ``x_shard`` holds this rank's points; ``n_total`` is the
    number of points over all ranks (summed with one more all-reduce when not
    given). Collective: every rank of ``group`` must call it."""
    if n_total is None:
        n_total = total_units(x_shard.shape[0], x_shard.device, group)
    if exch is not None:
        exch.zero_()  # the exchange vector accumulates (+=)
    exch = _lib.gmm_vjp_partial(x_shard, alpha, mu, q, l, gamma, m, prec, seed=seed, exch=exch, ws=ws,
                                status=status, stream=stream)
    combine(exch, group)
    return _lib.gmm_vjp_finalize(alpha, mu, q, l, n_total, exch, gamma, m, prec, seed=seed, d_alpha=d_alpha,
                                 d_mu=d_mu, d_q=d_q, d_l=d_l, out=out, ws=ws, status=status, stream=stream)


def reproj_vjp(cams, pts, obs_shard, w_shard, d_cams, d_pts, strat="auto", plan=None, ws=None, status=None,
               stream=None, group=None):
    """VJP of the reprojection residual over the observations of every rank:
    each rank scatters its shard into (d_cams, d_pts) (zeroed by the caller),
    then one all-reduce per array sums them. Collective."""
    _lib.reproj_vjp(cams, pts, obs_shard, w_shard, d_cams, d_pts, strat=strat, plan=plan, ws=ws, status=status,
                    stream=stream)
    combine(d_cams, group)
    combine(d_pts, group)
    return d_cams, d_pts


def gmm_vjp_from_host(x_host, alpha, mu, q, l, gamma=1.0, m=0, prec=_lib.PREC_FP32, seed=1.0, n_total=None,
                      chunk_points=1 << 18, d_alpha=None, d_mu=None, d_q=None, d_l=None, out=None, ws=None,
                      exch=None, staging=None, stream=None, copy_stream=None, group=None):
    """seed * grad f of the mixture over points held in host memory (pinned, so
    that copies run asynchronously): the points go to the device in chunks of
    ``chunk_points`` through two staging buffers, the copy of chunk c + 1 (on
    ``copy_stream``) overlapping gmm_vjp_partial on chunk c (on ``stream``);
    the chunks' exchange vectors accumulate, and the rank's sum is all-reduced
    and finished as in gmm_vjp. Device memory for the points stays at two
    chunks, whatever the number of points. ``staging``: two device float32
    buffers of at least chunk_points x D (allocated if not given); ``ws`` must
    serve a chunk. The first chunk is a quarter of chunk_points, which
    shortens the copy that nothing overlaps. Collective when ``group`` has more
    than one rank."""
    n, d = x_host.shape
    k = alpha.shape[0]
    dev = alpha.device
    chunk_points = max(128, (int(chunk_points) // 128) * 128)
    comp = torch.cuda.current_stream(dev) if stream is None else stream
    copy = torch.cuda.Stream(dev) if copy_stream is None else copy_stream
    if staging is None:
        c = min(chunk_points, n)
        staging = [torch.empty(c, d, dtype=torch.float32, device=dev) for _ in range(2)]
    if n_total is None:
        n_total = total_units(n, dev, group)
    e = _lib.gpa_gmm_exchange_len(d, k)
    if exch is None:
        exch = torch.zeros(e, dtype=torch.float64, device=dev)
    else:
        with torch.cuda.stream(comp):
            exch.zero_()
    if ws is None:
        ws = _lib.workspace(_lib.gpa_gmm_workspace_bytes(min(chunk_points, n), d, k, prec, 0), dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    copy.wait_stream(comp)  # staging buffers may still be read by earlier work on the compute stream
    # the first chunk is a quarter size: its copy is the one nothing overlaps
    first = max(128, (chunk_points // 4) // 128 * 128)
    bounds = [0] + list(range(min(first, n), n, chunk_points)) + [n]
    for c, (b0, b1) in enumerate(zip(bounds[:-1], bounds[1:])):
        slot = c % 2
        buf = staging[slot][:b1 - b0]
        if c >= 2:
            copy.wait_event(free[slot])  # chunk c - 2 is done with this buffer
        with torch.cuda.stream(copy):
            buf.copy_(x_host[b0:b1], non_blocking=True)
            copied[slot].record(copy)
        comp.wait_event(copied[slot])
        _lib.gmm_vjp_partial(buf, alpha, mu, q, l, gamma, m, prec, seed=seed, exch=exch, ws=ws, stream=comp)
        free[slot].record(comp)
    with torch.cuda.stream(comp):
        combine(exch, group)
    return _lib.gmm_vjp_finalize(alpha, mu, q, l, n_total, exch, gamma, m, prec, seed=seed, d_alpha=d_alpha,
                                 d_mu=d_mu, d_q=d_q, d_l=d_l, out=out, ws=ws, stream=comp)
