"""Plain FP64 CPU oracle for the Galactic-binary likelihood hot path.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run it. The product
package (``paper_2307_03763_gb300``) never imports it, and it imports nothing
from the product package: the two share no code, headers, tables or helpers.

Everything here is deliberately slow and obvious: PyTorch CPU ops in float64 /
complex128, direct sums, a naive O(N^2) DFT, Python loops for the Markov chain.
Each function cites the passage of Strub et al. (arXiv:2307.03763) it follows.
The paper cites, but does not print, the waveform and detector-response model
(Sec. III opening paragraph; Sec. III.G); ``gb.py`` writes that model out from
the physics of a plane wave crossing a rigid equal-arm triangle and
first-generation TDI, with every convention listed in its module docstring.

Modules
-------
gb      fast/slow template, naive DFT, window inner products, logL, gradient
mh      independence Metropolis-Hastings chain (Alg. 4, Eq. 13)
kde     reduced box and paired 2-D kernel-density proposals of the annealed
        posterior (Sec. III.G, Alg. 4)
noise   median-periodogram noise estimate of a segment (Sec. III.C)
brute   brute-force time-domain simulation of the same physics (no fast/slow
        split, exact delays), used only to pin ``gb`` against the physics
cpu_fft the oracle's likelihood with a radix-2 FFT in place of the naive DFT,
        timed as a second CPU baseline (not a checker of the GPU path)
"""
