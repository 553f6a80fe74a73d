"""TEST INFRASTRUCTURE: the oracle run in worker processes (a spawn pool), so that GPU tests can
check many independent node sets against it in parallel.  Imports nothing but numpy and the
oracle, so a freshly spawned worker starts quickly and touches no GPU."""


def assemble_job(args):
    """O.assemble(X, n, ell, m, delta) for one job; returns the arrays the parity checks use."""
    X, n, ell, m, delta = args
    from oracle import oracle as O
    r = O.assemble(X, n, ell, m, delta)
    out = {k: r[k] for k in ("row_ptr", "col", "val", "owner", "is_center", "lam_row", "nbr",
                             "d2")}
    out["n_near_tie"] = r["stats"]["n_near_tie"]
    return out


def pool(processes):
    """A spawn pool (safe after the parent has initialised CUDA)."""
    import multiprocessing
    return multiprocessing.get_context("spawn").Pool(processes)
