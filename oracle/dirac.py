"""Dirac matrices in the Euclidean Dirac basis (test infrastructure; see oracle/__init__).

The paper (Sec. 1, baryon operators) uses C gamma_5 and P_+- = (1 +- gamma_4)/2 without
fixing a basis.  Reading taken here: the Euclidean Dirac basis

    gamma_4 = diag(1, 1, -1, -1),  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
    gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4,  C = gamma_4 gamma_2.

Pinned in tests by C gamma_mu C^-1 = -gamma_mu^T, gamma_mu^2 = 1 and hermiticity.
"""
import numpy as np

_SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)
_Z = np.zeros((2, 2), dtype=np.complex128)

GAMMA = [np.block([[_Z, -1j * s], [1j * s, _Z]]) for s in _SIGMA]
GAMMA.append(np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128))
G1, G2, G3, G4 = GAMMA
G5 = G1 @ G2 @ G3 @ G4
C = G4 @ G2
CG5 = C @ G5
P_PLUS = 0.5 * (np.eye(4) + G4)
P_MINUS = 0.5 * (np.eye(4) - G4)
CG5_PPLUS = CG5 @ P_PLUS
CG5_PMINUS = CG5 @ P_MINUS
