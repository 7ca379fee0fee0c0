"""Oracle solves of the medium workload for the GPU parity tests, run in
worker processes (started with spawn, so no CUDA state is inherited) while
the test process drives the GPU.  Each worker regenerates the seeded system
itself, so only seeds and results cross the process boundary."""
import numpy as np

WORKLOAD = "medium"
XSEED, NSEED = 5, 6


def rhs(sys):
    """b = A x_true + noise, the right-hand side of the medium parity solves."""
    import oracle
    from paper_2212_11675_gb300 import gen
    return oracle.aprod1(sys, gen.x_true(sys, XSEED)) + gen.noise(sys, NSEED)


def perturbed(b, seed):
    """b with every entry moved by one unit of rounding (random sign): the
    oracle's own sensitivity to rounding, as in the smaller parity tests."""
    rng = np.random.default_rng(seed)
    return b * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=b.size))


def medium_solve(itmax, atol, btol, conlim, run_to_itmax, perturb_seed=None):
    import oracle
    from paper_2212_11675_gb300 import gen
    sys = gen.make(WORKLOAD)
    b = rhs(sys)
    if perturb_seed is not None:
        b = perturbed(b, perturb_seed)
    r = oracle.pc_lsqr(sys, b, itmax, atol, btol, conlim=conlim, run_to_itmax=run_to_itmax)
    return {k: r[k] for k in ("x", "se", "istop", "itn", "rnorm", "arnorm", "anorm", "acond",
                              "xnorm", "bnorm")}
