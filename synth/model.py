"""Model crystal, plane-wave spheres and the ground-state bundle.

Conventions (fixed here, used by every consumer of the bundle):

* ``lattice`` rows are the direct vectors a_i (bohr); reciprocal rows
  b_j = 2*pi*inv(A)^T with a_i.b_j = 2*pi*delta_ij; G = m @ B for Miller m.
* FFT grid n1 x n2 x n3, C order; grid point j <-> r_j = sum_i (j_i/n_i) a_i;
  Miller m lives at grid index (m mod n).
* Sphere S(p) = {m : |p + mB|^2 / 2 <= ecutwfc}, ordered by (|p+G|^2, m).
* Spinor coefficients c[s][g], sum |c|^2 = 1,
  psi_s(r_j) = Omega^{-1/2} sum_g c[s][g] exp(+i G.r_j).
* Local operators act as circular convolutions on the grid (this is how a
  plane-wave code realises V(r) psi(r)); the dense Hamiltonian built here uses
  exactly that convolution so that dense and FFT applications agree.
* Sister points (Sec. 5.2 of the paper, k, -k, k+-q, -k+-q) reduce to four
  Hamiltonians per k: side X uses H^(+) (exchange field +B, Eq. H0_k_plus_q),
  side Y uses H^(-) = T H_{-k} T^{-1} (field -B; spin-orbit is time-reversal
  invariant, so the nonlocal part is unchanged).
"""

from __future__ import annotations

import dataclasses
import numpy as np

HA_MEV = 27211.386245988  # 1 Hartree in meV

PAULI = np.array(
    [
        [[0, 1], [1, 0]],
        [[0, -1j], [1j, 0]],
        [[1, 0], [0, -1]],
    ],
    dtype=np.complex128,
)


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    return 2.0 * np.pi * np.linalg.inv(lattice).T


def cell_volume(lattice: np.ndarray) -> float:
    return float(abs(np.linalg.det(lattice)))


def grid_miller(fft) -> np.ndarray:
    """Centered Miller indices of every grid point, shape (Nr, 3), C order."""
    axes = [np.fft.fftfreq(n, d=1.0 / n).astype(np.int64) for n in fft]
    m1, m2, m3 = np.meshgrid(*axes, indexing="ij")
    return np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)


def miller_to_index(miller: np.ndarray, fft) -> np.ndarray:
    n1, n2, n3 = fft
    m = np.asarray(miller, dtype=np.int64)
    return ((m[:, 0] % n1) * n2 + (m[:, 1] % n2)) * n3 + (m[:, 2] % n3)


def sphere(p: np.ndarray, bvec: np.ndarray, ecut: float, fft) -> np.ndarray:
    """Miller indices of the plane-wave sphere at Bloch vector p (Cartesian)."""
    gmax = np.sqrt(2.0 * ecut) + np.linalg.norm(p)
    lat = 2.0 * np.pi * np.linalg.inv(bvec).T  # direct vectors
    bounds = [int(np.ceil(gmax * np.linalg.norm(lat[i]) / (2 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-b, b + 1) for b in bounds]
    m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    kin = 0.5 * np.sum((p[None, :] + m @ bvec) ** 2, axis=1)
    keep = kin <= ecut
    m, kin = m[keep], kin[keep]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], np.round(kin, 12)))
    m = m[order]
    for i, n in enumerate(fft):
        if m[:, i].min() < -(n // 2) or m[:, i].max() > (n - 1) // 2:
            raise ValueError(f"sphere does not fit the FFT box along axis {i}")
    return m.astype(np.int32)


@dataclasses.dataclass
class KBChannel:
    """One Kleinman-Bylander projector: Gaussian radial part times a real harmonic."""

    rc: float
    harm: str  # 's', 'px', 'py', 'pz'


@dataclasses.dataclass
class Atom:
    tau: np.ndarray  # Cartesian position (bohr)
    channels: list  # list[KBChannel]
    dmat: np.ndarray  # (nch, nch) real symmetric coupling (Ha)
    lam_so: float  # spin-orbit strength on the p block (Ha)
    so_mode: str  # 'full' (L.sigma) or 'z' (L_z sigma_z)


def projector_values(p: np.ndarray, miller: np.ndarray, bvec: np.ndarray, omega: float,
                     atoms: list) -> np.ndarray:
    """beta_{a,i}(p+G) = Omega^{-1/2} N_i g(|p+G|) Y_i(p+G) exp(-i (p+G).tau_a)."""
    kg = p[None, :] + miller.astype(np.float64) @ bvec
    k2 = np.sum(kg * kg, axis=1)
    rows = []
    for at in atoms:
        phase = np.exp(-1j * (kg @ at.tau))
        for ch in at.channels:
            g = np.exp(-0.5 * k2 * ch.rc ** 2)
            if ch.harm == "s":
                y = np.ones_like(k2)
                norm = np.sqrt(8.0 * np.pi ** 1.5 * ch.rc ** 3)
            else:
                y = kg[:, "xyz".index(ch.harm[1])]
                norm = np.sqrt(16.0 * np.pi ** 1.5 * ch.rc ** 5)
            rows.append(norm * g * y * phase / np.sqrt(omega))
    return np.array(rows, dtype=np.complex128)


def l_matrix_cartesian() -> np.ndarray:
    """(L_k)_{ij} = -i eps_{kij} on the real p harmonics (p_x, p_y, p_z)."""
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    return -1j * eps


def atom_dmatrix(at: Atom) -> np.ndarray:
    """D_a = d (x) I_2 + lam_so (L.sigma)/2 on each radial channel's p block.

    Index (i, s) -> 2*i + s.  Hermitian and time-reversal invariant.
    """
    nch = len(at.channels)
    dm = np.kron(at.dmat.astype(np.complex128), np.eye(2))
    lmat = l_matrix_cartesian()
    for i, ci in enumerate(at.channels):
        for j, cj in enumerate(at.channels):
            if ci.harm == "s" or cj.harm == "s" or ci.rc != cj.rc:
                continue
            a, b = "xyz".index(ci.harm[1]), "xyz".index(cj.harm[1])
            if at.so_mode == "z":
                blk = lmat[2, a, b] * PAULI[2]
            else:
                blk = sum(lmat[k, a, b] * PAULI[k] for k in range(3))
            dm[2 * i:2 * i + 2, 2 * j:2 * j + 2] += 0.5 * at.lam_so * blk
    assert np.allclose(dm, dm.conj().T)
    return dm


def block_diag(mats) -> np.ndarray:
    n = sum(m.shape[0] for m in mats)
    out = np.zeros((n, n), dtype=np.complex128)
    o = 0
    for m in mats:
        k = m.shape[0]
        out[o:o + k, o:o + k] = m
        o += k
    return out


@dataclasses.dataclass
class GroundState:
    """The ground-state bundle (all host arrays, FP64)."""

    lattice: np.ndarray  # (3,3) rows a_i
    fft: tuple
    ecutwfc: float
    nk: int
    kpts: np.ndarray  # (nk,3) Cartesian
    q: np.ndarray  # (3,) Cartesian
    wk: np.ndarray  # (nk,)
    nocc: int
    npwx: int
    npw_k: np.ndarray  # (nk,)
    npw_kq: np.ndarray  # (nk,)
    miller_k: np.ndarray  # (nk,npwx,3) int32
    miller_kq: np.ndarray  # (nk,npwx,3) int32
    evals: np.ndarray  # (2,nk,nocc)  sides X,Y at k
    evals_kq: np.ndarray  # (2,nk,nocc) sides X,Y at k+q
    coeff_k: np.ndarray  # (2,nk,nocc,2,npwx) complex
    coeff_kq: np.ndarray  # (2,nk,nocc,2,npwx) complex
    vloc: np.ndarray  # (Nr,)
    bfield: np.ndarray  # (3,Nr)
    n0: np.ndarray  # (Nr,)
    m0: np.ndarray  # (3,Nr)
    nproj: int
    beta_kq: np.ndarray  # (nk,nproj,npwx) complex
    dnl: np.ndarray  # (2nproj,2nproj) complex, index 2*i+s
    kernel_mask: int = 3  # bit0 Hartree, bit1 XC; 0 = independent-particle mode
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nr(self) -> int:
        return int(np.prod(self.fft))

    @property
    def omega(self) -> float:
        return cell_volume(self.lattice)

    @property
    def br_shape(self):
        return (2, self.nk, self.nocc, 2, self.npwx)

    def with_kernel_mask(self, mask: int) -> "GroundState":
        return dataclasses.replace(self, kernel_mask=int(mask))

    def save(self, path: str) -> None:
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self) if f.name != "meta"}
        d["fft"] = np.array(self.fft)
        np.savez_compressed(path, **d)

    @staticmethod
    def load(path: str) -> "GroundState":
        z = np.load(path)
        kw = {k: z[k] for k in z.files}
        kw["fft"] = tuple(int(v) for v in kw["fft"])
        for k in ("ecutwfc",):
            kw[k] = float(kw[k])
        for k in ("nk", "nocc", "npwx", "nproj", "kernel_mask"):
            kw[k] = int(kw[k])
        return GroundState(**kw)
