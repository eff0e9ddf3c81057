"""CPU oracle of IVF-RaBitQ (test infrastructure).

Plain, slow, obviously-correct numpy code that the CUDA library is checked
against. It shares no code with the CUDA path and neither imports the other.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` may import it.

Pins (the tests under ``tests/test_oracle_*.py``) tie each function to what
the paper and mathematics fix: Philox known-answer vectors, orthogonality of
P, the alpha identity of Eq. 3, the exact integer identity behind the
bit-plane estimator, unbiasedness of Eq. 4 over random rotations, the closed
form of Eq. 5, quantisation error bounds, and exact brute-force kNN in the
nprobe = nList limit. Every function here has at least one such pin.
"""
from . import philox, rabitq  # noqa: F401
