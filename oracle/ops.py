"""Local operators for the oracle (Sec. 3.1 of the paper: spin and boson sets).

All operators are real float64 matrices indexed ``[out, in]`` (bra, ket).
The y-components of spins are imaginary; models here only use products in
which the imaginary unit cancels, so the oracle carries ``iSy`` (a real
antisymmetric matrix) instead of ``Sy``:  Sy (x) Sy = -(iSy) (x) (iSy).
"""
import numpy as np


def spin_half():
    """Pauli matrices and spin-1/2 operators S = sigma/2 in the basis (up, down)."""
    sx = np.array([[0.0, 1.0], [1.0, 0.0]])
    sz = np.array([[1.0, 0.0], [0.0, -1.0]])
    isy = np.array([[0.0, 1.0], [-1.0, 0.0]])  # i * sigma_y
    eye = np.eye(2)
    return {
        "id": eye,
        "sigma_x": sx,
        "sigma_z": sz,
        "i_sigma_y": isy,
        "Sx": sx / 2,
        "Sz": sz / 2,
        "iSy": isy / 2,
        "Sp": np.array([[0.0, 1.0], [0.0, 0.0]]),  # S+ |down> = |up>
        "Sm": np.array([[0.0, 0.0], [1.0, 0.0]]),
    }


def spin_one():
    """Spin-1 operators in the basis (m=+1, 0, -1)."""
    r2 = np.sqrt(2.0)
    sp = np.array([[0.0, r2, 0.0], [0.0, 0.0, r2], [0.0, 0.0, 0.0]])
    sm = sp.T.copy()
    sx = (sp + sm) / 2
    isy = (sp - sm) / 2  # i*Sy = i * (S+ - S-)/(2i)
    sz = np.diag([1.0, 0.0, -1.0])
    return {"id": np.eye(3), "Sx": sx, "iSy": isy, "Sz": sz, "Sp": sp, "Sm": sm}


def boson(nmax):
    """Truncated boson operators b, b^dagger, n on occupations 0..nmax."""
    d = nmax + 1
    b = np.zeros((d, d))
    for n in range(1, d):
        b[n - 1, n] = np.sqrt(n)
    bd = b.T.copy()
    num = np.diag(np.arange(d, dtype=np.float64))
    return {"id": np.eye(d), "b": b, "bd": bd, "n": num}
