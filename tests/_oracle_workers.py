"""Oracle work for spawned worker processes in the GPU tests (the worker
function must live in an importable module, not in a test file)."""
import workloads
from oracle import mps


def oracle_state(args):
    """(workload name, row, storage) -> (state rounded to the storage
    precision, bond dimensions), built by the oracle."""
    name, row, store = args
    w = workloads.BY_NAME[name]()
    r = mps.build_mps(w.X[row], w.d, w.reps, w.gamma, w.chi_max, w.eps)
    return mps.round_sites(r.sites, store), r.bond_dims
