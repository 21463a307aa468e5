"""Per-solve comparison of a GPU step with the oracle's step (test helper).

Both sides run the same algorithm (x0 = 0, FGMRES(m), CGS2, the same
preconditioner), so a solve is compared iterate against iterate.  When the
two stop one Krylov iteration apart (rounding moves the stopping test), the
oracle step is run again with every FGMRES stopped after exactly the GPU's
iteration count (rtol = atol = 0, maxit = that count): its result for that
solve is the Arnoldi iterate the GPU returned, and is compared at the same
tolerance.  The solves of one step are independent given the step-k state
(all coefficients at t_k, Sec. 3), so stopping the others early does not
change the solve under comparison."""
import numpy as np

SOLVE_TOL = 1e-9        # FP64 GPU vs FP64 oracle, per solve (relative L2)

GROUPS = [("ch_p", (("phi", 0), ("mu", 0))), ("ch_N", (("phi", 1), ("mu", 1))), ("ch_s", (("phi", 2), ("mu", 2))),
          ("ac", (("Phi_v", None),)), ("ns", (("v", None), ("p", None)))]


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def fields(state, keys):
    return np.concatenate([np.ravel(state[k] if i is None else state[k][i]) for k, i in keys])


def oracle_at_iterations(make_oracle, params, state, iters):
    """The oracle step with every FGMRES stopped after exactly `iters`
    iterations."""
    p = dict(params, rtol=0.0, atol=0.0, maxit=int(iters))
    if p.get("ns_rtol", 0.0) > 0:
        p.update(ns_rtol=0.0, ns_atol=0.0)
    return make_oracle(p).step(state)[0]


def compare_solves(got, info, ref, rinfo, state, params, make_oracle, names=None, tol=SOLVE_TOL, where=""):
    """Every FGMRES solve of a GPU step against the oracle: converged,
    iterations within +-1, and the values within tol (against the oracle
    iterate at the GPU's count when the counts differ).  Returns the names
    that needed the re-run."""
    rerun = []
    for name, keys in GROUPS:
        if names is not None and name not in names:
            continue
        gi, ri = info[name]["iters"], rinfo[name]["iters"]
        assert info[name]["converged"], (where, name, info[name])
        assert abs(gi - ri) <= 1, (where, name, info[name], rinfo[name])
        r = ref
        if gi != ri:
            r = oracle_at_iterations(make_oracle, params, state, gi)
            rerun.append(name)
        e = rel(fields(got, keys), fields(r, keys))
        assert e <= tol, (where, name, gi, ri, e)
    return rerun
