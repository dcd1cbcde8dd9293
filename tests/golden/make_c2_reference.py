"""Writes tests/golden/c2_xref.npz: the oracle's solution of the 128 x 128
workload (180 views x 182 bins, sqrt(lambda) = 0.05, noisy sinograms I0 = 1e4)
for the first K phantoms, by the paper's in-core route of Sec. 2.1 (LAPACK
dgeqrf + dormqr + dtrtrs on the oracle's dense A~).  Calls only oracle/ and
the seeded input generators.  Run:  python tests/golden/make_c2_reference.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2412_07631_b300 import synth  # noqa: E402

NS, NV, NB, SL, K, SEED = 128, 180, 182, 0.05, 16, 4321


def inputs():
    g = O.Geometry(NS, NV, NB, sqrt_lambda=SL)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(NS, K, 10)
    B = synth.poisson_sinogram(O.forward(csr, X), NS, 1e4, seed=SEED)
    return g, csr, X, B


def digest(B):
    return hashlib.sha256(np.ascontiguousarray(B).tobytes()).hexdigest()


def main():
    g, csr, X, B = inputs()
    A = O.dense_system(g, csr)
    Xo, R = O.lapack_qr_solve(g, A, B, overwrite=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_xref.npz")
    np.savez_compressed(out, xref=Xo, b_sha256=digest(B), rdiag=np.abs(np.diag(R)))
    print(out, Xo.shape)


if __name__ == "__main__":
    main()
