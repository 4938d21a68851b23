"""Oracle runs for process pools (spawned workers import this module, which
loads neither torch nor the CUDA library)."""
from oracle import oracle as O
from paper_2411_00991_gb300 import synth


def small_chain_mean(H, W, L, seed, burn_in, refresh_every, T, chain):
    """Posterior mean of one oracle chain of ``synth.small_problem``."""
    p = synth.small_problem(H=H, W=W, L=L, seed=seed, burn_in=burn_in, refresh_every=refresh_every)
    r = O.Oracle(p, chain=chain).run(T)
    return r["sum"] / r["n_sum"]


def log_posterior_fft(prob, rho):
    """Eq. 9 of one state (the oracle's evaluator for large frames)."""
    return O.Oracle(prob).log_posterior_fft(rho)


def log_posterior(prob, rho):
    """Eq. 9 of one state (the oracle's definitional evaluator)."""
    return O.Oracle(prob).log_posterior(rho)
