"""The exchange of a multi-rank VMC step: chains split over processes, one per GPU.

Markov chains are independent, so each rank samples its own chains with the same
parameters and the step needs one exchange, two SUM all-reduces of FP64 buffers the
library's kernels wrote (no arithmetic here):

1. the additive moments of each rank's statistics (nqs_stats_moments); the library turns
   their sum into the pooled statistics (nqs_stats_finalize), so every rank holds the
   global E and sample count;
2. each rank's force share (nqs_force_share), centred on that global E and divided by the
   global count; the shares sum to the force of the pooled samples (App. I, Eq. forces).

Centring each rank on its own E_r instead would drop the term sum_r (E - E_r) sum_{x in r} O(x).
"""
import torch.distributed as dist


def exchange_stats(ctx, moments, stats, group=None):
    """Sums `moments` [8] over the ranks in place and writes the pooled statistics to `stats` [5]."""
    dist.all_reduce(moments, op=dist.ReduceOp.SUM, group=group)
    ctx.stats_finalize(moments, stats)


def exchange_force(force_share, group=None):
    """Sums the ranks' force shares [P] in place: the force of the pooled samples."""
    dist.all_reduce(force_share, op=dist.ReduceOp.SUM, group=group)
