"""Writes tests/golden/c4_grad.npz: the oracle's FP64 gradient of the
differentiation workload's loss with respect to the sinograms, for a few
sampled slices.

Workload: the 128 x 128 geometry (180 views x 182 bins, sqrt(lambda) = 0.05),
a batch of 256 ten-ellipse phantoms (seeds 1234..1489), Poisson sinograms at
I0 = 1e4 (noise seed 23), loss L = ||X - X_phantom||_F^2 / (n k) with k = 256.

The reconstruction is x = R^-1 Q1^T b~ (Sec. 2 Eq. 3), so with
g = dL/dx = 2 (x - x_phantom) / (n k) the gradient is
dL/db = [Q [R^-T g; 0]]_{0:m}: the transpose of each step of Eq. 3 taken in
reverse order.  Every step is a LAPACK call on the oracle's dense FP64 A~ (the
paper's in-core route of Sec. 2.1, oracle.lapack_qr_gradient): dgeqrf once;
dormqr('T') and dtrtrs for x, then dtrtrs (transposed) and dormqr('N') for
the gradient.

Calls only oracle/ and the seeded input generators.
Run:  python tests/golden/make_c4_gradient.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2412_07631_b300 import synth  # noqa: E402

NS, NV, NB, SL, K, SEED = 128, 180, 182, 0.05, 256, 23
SLICES = (0, 1, 85, 170, 254, 255)


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
    S = list(SLICES)
    A = O.dense_system(g, csr)
    grad, xref = O.lapack_qr_gradient(g, A, np.asfortranarray(B[:, S]), X[:, S], K, overwrite=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_grad.npz")
    np.savez_compressed(out, grad_b=np.ascontiguousarray(grad), slices=np.array(S), xref=xref,
                        b_sha256=digest(B))
    print(out, grad.shape)


if __name__ == "__main__":
    main()
