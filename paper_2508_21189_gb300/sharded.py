"""Row-sharded sketches over several processes, one GPU each.

The sketch of a tall A is additive over row blocks: with A split into row blocks A_g (rows
[r_g, r_{g+1})), S A = sum_g S[:, r_g:r_{g+1}] A_g, and the same holds for the SRTT once the blocks
start on 2048-row boundaries (H_N = H_{N/2048} (x) H_2048).  The paper states the sketch cost
O(zeta nnz(A)) (Sec. 3.2), which is additive over the blocks; the only exchange is one d x k sum.

Each rank computes its partial in the library (rsk_sparse_sign_apply_rows / rsk_srtt_apply_rows);
this module gathers the partials in rank order over the process group and sums them in rank order
with the library's ordered sum (rsk_sketch_sum_partials), so the result is the same on every rank
and for every run with the same world size.  Only the partition and the collective live here.
"""
import torch
import torch.distributed as dist


def row_partition(n, world, align=1):
    """Row blocks (row0, rows) of an n-row matrix over `world` ranks, every row0 a multiple of
    `align` (2048 for the SRTT); blocks differ in size by at most `align` rows.  A rank may get an
    empty block only when n < world * align."""
    if n < 1 or world < 1 or align < 1:
        raise ValueError("need n, world, align >= 1")
    units = -(-n // align)
    out = []
    for g in range(world):
        u0, u1 = units * g // world, units * (g + 1) // world
        r0, r1 = min(n, u0 * align), min(n, u1 * align)
        out.append((r0, r1 - r0))
    return out


def gather_partials(partial, group=None):
    """[world, d, k] tensor of every rank's partial, in rank order (all ranks get all of them)."""
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(partial) for _ in range(world)]
    dist.all_gather(bufs, partial.contiguous(), group=group)
    return torch.stack(bufs)


def reduce_partials(partial, sum_partials, group=None):
    """The whole sketch on every rank: the partials gathered in rank order and summed in rank
    order by `sum_partials` ([world, d, k] -> [d, k]; the library's rsk_sketch_sum_partials on the
    GPU path)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return sum_partials(partial.unsqueeze(0))
    return sum_partials(gather_partials(partial, group))


def sparse_sign_apply(A_local, row0, d, zeta, seed, group=None, out_dtype=torch.float32):
    """S A for a row-sharded A: this rank holds rows row0 .. row0 + n_local - 1 (A_local on its GPU)."""
    import paper_2508_21189_gb300 as rsk
    part = rsk.rsk_sparse_sign_apply_rows(A_local, row0, d, zeta, seed, out_dtype=out_dtype)
    return reduce_partials(part, rsk.rsk_sketch_sum_partials, group)


def srtt_apply(A_local, row0, n_total, d, seed, group=None, out_dtype=torch.float32):
    """SRTT of a row-sharded A (N = n_total rows; row0 a multiple of 2048 on every rank)."""
    import paper_2508_21189_gb300 as rsk
    part = rsk.rsk_srtt_apply_rows(A_local, row0, n_total, d, seed, out_dtype=out_dtype)
    return reduce_partials(part, rsk.rsk_sketch_sum_partials, group)
