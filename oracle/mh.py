"""Independence Metropolis-Hastings chain built from precomputed values, plain FP64.

TEST INFRASTRUCTURE (see the package docstring).

Sec. III.G: because the proposal g does not depend on the chain state, every
log-likelihood of the n proposals is computed first (in parallel) and the chain
is built afterwards by one sequential scan (Alg. 4).  The acceptance probability
is Eq. 13,  P = min(1, [L_p/L_c * g(theta_c)/g(theta_p)]^(1/T)).

Readings
--------
M1  Temperature: by default the exponent 1/T acts on the likelihood ratio only,
        Delta = (l_i - l_c)/T + (log g_c - log g_i),
    which is the Metropolis-Hastings rule for the tempered target L^(1/T).
    ``literal=True`` applies 1/T to the whole bracket as printed in Eq. 13,
        Delta = ((l_i - l_c) + (log g_c - log g_i))/T.
    Both are evaluated through one weight per proposal, in this rounding order:
        default   w_i = l_i/T - log g_i,   Delta = w_i - w_c
        literal   v_i = l_i - log g_i,     Delta = (v_i - v_c)/T
    (mathematically the same quantities).  The two agree bit for bit at T = 1.
M2  "With probability alpha" is decided by a uniform variate u_i in (0, 1)
    passed in as its logarithm: accept iff log u_i < min(0, Delta).  Working
    in logs needs only +, -, / and a comparison, so two IEEE implementations
    that use the same operation order take identical decisions.
M3  The chain has n entries: chain[0] = 0 (theta_1 is the start state) and
    chain[i] is the state index after step i.  The paper's list is chain[1:].
M4  logL = -inf (a proposal outside the prior) is never accepted; a NaN
    Delta (both -inf) counts as a rejection.
"""
import math


def mh_independence(logL, log_g, log_u, temperature, literal=False):
    """One chain over n precomputed proposals (Alg. 4 inner loop, Eq. 13).

    logL, log_g, log_u: sequences of n floats; temperature: float > 0.
    Returns (chain, n_accept) with chain a list of n ints.
    """
    n = len(logL)
    if n == 0:
        return [], 0
    c = 0
    chain = [0]
    n_accept = 0
    T = float(temperature)
    if literal:
        w = [float(logL[i]) - float(log_g[i]) for i in range(n)]
    else:
        w = [float(logL[i]) / T - float(log_g[i]) for i in range(n)]
    for i in range(1, n):
        delta = (w[i] - w[c]) / T if literal else w[i] - w[c]
        if math.isnan(delta):
            accept = False
        else:
            accept = float(log_u[i]) < min(0.0, delta)
        if accept:
            c = i
            n_accept += 1
        chain.append(c)
    return chain, n_accept


def mh_independence_batch(logL, log_g, log_u, temperature, literal=False):
    """Independent chains of Alg. 4, one per row: inputs (n_chains, n);
    temperature (n_chains,)."""
    chains, acc = [], []
    for r in range(len(logL)):
        ch, a = mh_independence(logL[r], log_g[r], log_u[r], temperature[r], literal)
        chains.append(ch)
        acc.append(a)
    return chains, acc
