"""Isolated partitions of one simulation and the merge of their species.

The Independent algorithm traces every sampled individual's lineage from
(seed, location, time) alone, so the sample of one simulation can be split
into parts that run with no communication at all (the paper's
IsolatedIndividuals and IsolatedLandscape strategies, section "The
Independent Algorithm" of its parallelisation chapter, and section
"Biodiversity Simulation Limit Analysis", where 7.1e10 individuals ran as
independent partitions).
Lineages of different parts that meet are simulated once in each part; an
individual's speciation key is the same in its part as in the whole
simulation.  The one exchange is at the end: the parts' distinct speciation
keys are gathered and ranked into global species identities.

Argument marshalling and the exchange only: sampling, the simulation, the
sort/unique and the ranks run in the library's kernels (sim_sample_partition,
ind_keys_unique, ind_keys_rank).  The exchange is an all-gather of each
part's distinct keys over torch.distributed (NCCL between GPUs, gloo on CPU
tensors), 16 bytes per distinct key and part.
"""
from . import PARTITION_INDIVIDUALS, PARTITION_LANDSCAPE, keys_rank, keys_unique  # noqa: F401


def run_part(sim, part, n_parts, scheme=PARTITION_LANDSCAPE, fraction=1.0, sample_seed=0, round_budget=0):
    """sample part `part` of n_parts of `sim`'s individuals and run it to the
    end; returns the part's speciation keys per individual (device tensors,
    in the whole sample's order restricted to the part)"""
    sim.sample_partition(part, n_parts, scheme, fraction, sample_seed)
    if not sim.run(round_budget):
        raise RuntimeError("the partition's run did not finish within its round budget")
    return sim.species_keys(device=True)


def gather_keys(pg, key_loc, key_time):
    """all ranks' keys: an all-gather of variable-length (location, time)
    key sets over the process group `pg` (torch.distributed); returns the
    concatenation in rank order, on the inputs' device"""
    import torch
    dev = key_loc.device
    n = torch.tensor([key_loc.numel()], dtype=torch.int64, device=dev)
    world = pg.get_world_size()
    sizes = [torch.zeros_like(n) for _ in range(world)]
    pg.all_gather(sizes, n)
    sizes = [int(x.item()) for x in sizes]
    m = max(sizes + [1])
    # uint64 travels as int64 (the same bits)
    pad = torch.zeros(2, m, dtype=torch.int64, device=dev)
    pad[0, :key_loc.numel()] = key_loc.view(torch.int64)
    pad[1, :key_time.numel()] = key_time.view(torch.int64)
    bufs = [torch.empty_like(pad) for _ in range(world)]
    pg.all_gather(bufs, pad)
    kl = torch.cat([b[0, :k] for b, k in zip(bufs, sizes)]).view(torch.uint64)
    kt = torch.cat([b[1, :k] for b, k in zip(bufs, sizes)]).view(torch.uint64)
    return kl, kt


def merge_species(key_loc, key_time, pg=None, part_keys=None):
    """global species identities of this part's individuals from its keys
    (device tensors): the part's distinct keys, every part's distinct keys
    (gathered over `pg`, or given as part_keys = [(loc, time), ...] when all
    parts ran on this device), their global distinct set, and each
    individual's rank in it.  Returns (identities, species count)."""
    import torch
    ul, ut = keys_unique(key_loc, key_time)
    if pg is not None:
        al, at = gather_keys(pg, ul, ut)
    elif part_keys is not None:
        uniq = [keys_unique(l, t) for l, t in part_keys]
        al = torch.cat([u[0] for u in uniq])
        at = torch.cat([u[1] for u in uniq])
    else:
        al, at = ul, ut
    gl, gt = keys_unique(al, at)
    return keys_rank(key_loc, key_time, gl, gt), int(gl.numel())
