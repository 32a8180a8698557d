"""Assignment of independent batched instances to ranks.

Batched instances share nothing, so a multi-GPU run shards them by instance with no
collective in the data path: each rank steps its own subset on its own GPU and only the
timings and update counts are reduced at the end.  The subsets come from greedy
longest-processing-time scheduling (largest cost first, each onto the currently lightest
rank) on the per-step cost model N_x * N_v * (k + 2): a step of an instance sweeps its
N_x * N_v cell-directions k times in SI-DSA and twice more in the b~ / f sweep (Sec. 4's sweep
count), k being the expected SI iterations per step.  Greedy LPT is within a factor
4/3 - 1/(3m) of the best makespan on m ranks (Graham's bound).  Every rank computes the same
assignment from the same inputs (ties go to the lower index), so no exchange is needed.
"""


def instance_cost(ncell, n_dirs, iterations=3.0):
    """Expected cell-direction updates of one implicit step."""
    return float(ncell) * float(n_dirs) * (float(iterations) + 2.0)


def lpt_partition(costs, nranks):
    """Indices of `costs` per rank (each list ascending); every index on exactly one rank."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    loads = [0.0] * nranks
    parts = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += float(costs[i])
    return [sorted(p) for p in parts]


def workload_directions(wl):
    """Direction count of a workload's quadrature description."""
    q = wl.quadrature
    if q[0] == "gl":
        return int(q[1])
    if q[0] == "cl_hemi":
        return int(q[1]) * int(q[2]) // 2
    raise ValueError(f"unknown quadrature {q!r}")


def shard(workloads, rank, world, iterations=3.0):
    """(indices, workloads) of `rank`'s share of the batch."""
    costs = [instance_cost(w.ncell, workload_directions(w), iterations) for w in workloads]
    idx = lpt_partition(costs, world)[rank]
    return idx, [workloads[i] for i in idx]
