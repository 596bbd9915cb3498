"""Workload definitions and the ground-state bundle builder.

Configs (seed 1000 + id unless given):

* C0  -- oracle micro case: simple cubic a=6, 12^3 grid, ~70 PW per spinor
  component, Gamma only, 4 occupied bands, 1 atom x {p_x, p_y} with
  lambda L_z sigma_z / 2, q = (0.1,0,0) 2pi/a.
* C0K -- C0 with a 2-point k grid (exercises the k sums and distinct spheres).
* C1  -- simple cubic a=8, 16^3, ~300 PW, Gamma, 8 bands, 2 atoms x 2 projectors.
* C2  -- hexagonal a=13, c=30 (vacuum slab), 36x36x96, ~5000 PW, 4x4 k grid,
  40 bands, 8 atoms x 8 projectors (2 radial x {s,p}) with full L.sigma.
* C3  -- hexagonal a=13, c=38, 45x45x144, ~12000 PW, 8x8 k grid, 70 bands.
* C5  -- the batched form's cell: C3's on a 4x4 k grid, a cutoff per q-point.

The hexagonal atoms sit at the in-plane fractional positions of a CrI3
monolayer (2 "Cr" + 6 "I" sites) with the layer centred in the cell.
Units: Hartree atomic units; q is given in 2pi/a along Cartesian x.
"""

from __future__ import annotations

import dataclasses
import numpy as np
import scipy.fft

from .model import (Atom, GroundState, KBChannel, PAULI, atom_dmatrix, block_diag,
                    cell_volume, miller_to_index, projector_values, reciprocal, sphere)
from .hamiltonian import HamiltonianFFT, dense_hamiltonian
from .eigensolver import dense_lowest, lobpcg


@dataclasses.dataclass
class Config:
    name: str
    lattice: np.ndarray
    fft: tuple
    ecut: float
    kgrid: tuple
    nocc: int
    q_2pi_a: tuple
    kind: str  # 'cubic' or 'hex'
    v_sigma: float = 0.1
    v_gcut: float = 3.0
    b0: float = 0.2
    b_noncollinear: float = 0.5
    lam_so_scale: float = 1.0
    seed: int = 1000
    alat: float = 1.0
    natom: int = 0              # cubic cells: atoms (0: one for C0*, two otherwise)
    well_depth: float = 0.0     # Gaussian wells -V exp(-|r - R|^2 / (2 w^2)) added to v_loc,
    well_width: float = 1.0     # centred at R = first atom + each of well_shifts (bohr)
    well_shifts: tuple = ((0.0, 0.0, 0.0),)


def _cubic(a):
    return np.diag([a, a, a]).astype(np.float64)


def _hex(a, c):
    return np.array([[a, 0, 0], [-0.5 * a, 0.5 * np.sqrt(3) * a, 0], [0, 0, c]], dtype=np.float64)


CONFIGS = {
    "C0": Config("C0", _cubic(6.0), (12, 12, 12), 3.6, (1, 1, 1), 4, (0.1, 0, 0), "cubic",
                 seed=1000, alat=6.0),
    "C0K": Config("C0K", _cubic(6.0), (12, 12, 12), 3.6, (1, 2, 1), 4, (0.1, 0, 0), "cubic",
                  seed=1010, alat=6.0),
    "C0F": Config("C0F", _cubic(6.0), (20, 15, 18), 3.6, (1, 2, 1), 4, (0.1, 0.05, 0), "cubic",
                  seed=1020, alat=6.0),
    "C1": Config("C1", _cubic(8.0), (16, 16, 16), 5.3, (1, 1, 1), 8, (0.1, 0, 0), "cubic",
                 seed=1001, alat=8.0),
    "C2": Config("C2", _hex(13.0, 30.0), (36, 36, 96), 8.3, (4, 4, 1), 40, (0.125, 0, 0), "hex",
                 seed=1002, alat=13.0),
    "C3": Config("C3", _hex(13.0, 38.0), (45, 45, 144), 12.7, (8, 8, 1), 70, (0.125, 0, 0), "hex",
                 seed=1003, alat=13.0),
    # the batched form's cell: C3's cell and grid on a 4x4 k grid; each q-point of the
    # batch sets its own cutoff (c5_ecut) so that the k+q spheres hold 10000-13000 PW
    "C5": Config("C5", _hex(13.0, 38.0), (45, 45, 144), 12.7, (4, 4, 1), 70, (0.0625, 0, 0),
                 "hex", seed=1005, alat=13.0),
    # a spontaneously magnetic model for the Goldstone check: two electrons per cell bound
    # in two deep Gaussian wells 3.5 bohr apart, polarised in parallel by the
    # self-consistent Slater exchange without an external field; the atom's p projectors
    # (lambda L_z sigma_z / 2, lambda = 0.9 Ha) sit 0.7 bohr off the first well so that
    # spin-orbit coupling reaches the occupied states.  The cutoff lies halfway between
    # two shells of |G|^2 (2 ecut = 12.5 (2 pi / a)^2), so the k+q spheres equal the k
    # sphere for |q| < 0.06 (2 pi / a) and L changes smoothly with q there.
    "CG": Config("CG", _cubic(8.0), (16, 16, 16), 3.8553, (1, 1, 1), 2, (0.01, 0, 0), "cubic",
                 v_sigma=0.02, b_noncollinear=0.0, lam_so_scale=3.0, seed=1007, alat=8.0,
                 natom=1, well_depth=3.0, well_width=1.0,
                 well_shifts=((0.7, 0.0, 0.0), (-2.8, 0.0, 0.0))),
}


def c5_ecut(m: int, nq: int = 6) -> float:
    """Cutoff (Ha) of q-point m = 1..nq of the batched form: plane waves per spinor
    component from 10000 (m = 1) to 13000 (m = nq) in equal steps, using Np ~ ecut^(3/2)
    from C3's ~12000 at 12.7 Ha."""
    npw = 10000.0 + 3000.0 * (m - 1) / max(nq - 1, 1)
    return 12.7 * (npw / 12000.0) ** (2.0 / 3.0)

# CrI3 monolayer sites, crystal coordinates (in-plane) and layer height offsets
# relative to the Cr plane in bohr (c = 37.38 bohr in the reference structure).
_CRI3_FRAC = np.array([
    [0.6666667, 0.3333333, 0.6667240],
    [0.0000000, 0.0000000, 0.6666093],
    [0.9788986, 0.6665119, 0.7464249],
    [0.6876134, 0.0211013, 0.7464249],
    [0.3334880, 0.3123867, 0.7464249],
    [0.6877680, 0.6668213, 0.5869084],
    [0.9790533, 0.3122319, 0.5869084],
    [0.3331787, 0.0209467, 0.5869084],
])


def _atoms(cfg: Config, rng) -> list:
    lat = cfg.lattice
    if cfg.kind == "cubic":
        natom = cfg.natom or (1 if cfg.name.startswith("C0") else 2)
        atoms = []
        for a in range(natom):
            frac = rng.uniform(0.2, 0.8, size=3)
            chans = [KBChannel(1.0, "px"), KBChannel(1.0, "py")]
            atoms.append(Atom(frac @ lat, chans, np.diag([1.2, 1.2]) * (1 + 0.2 * a),
                              0.3 * cfg.lam_so_scale, "z"))
        return atoms
    atoms = []
    c = lat[2, 2]
    for a, f in enumerate(_CRI3_FRAC):
        z = (f[2] - 0.6666667) * 37.38 + 0.5 * c
        tau = f[0] * lat[0] + f[1] * lat[1] + np.array([0, 0, z])
        heavy = a >= 2
        rcs = (0.9, 1.5) if heavy else (0.7, 1.2)
        chans = [KBChannel(rc, h) for rc in rcs for h in ("s", "px", "py", "pz")]
        d = np.zeros((8, 8))
        ds = np.array([[1.5, 0.3], [0.3, -0.6]])
        dp = np.array([[0.9, 0.2], [0.2, -0.4]])
        for hi in range(4):
            blk = ds if hi == 0 else dp
            for r1 in range(2):
                for r2 in range(2):
                    d[r1 * 4 + hi, r2 * 4 + hi] = blk[r1, r2]
        lam = (0.3 if heavy else 0.05) * cfg.lam_so_scale
        atoms.append(Atom(tau, chans, d, lam, "full"))
    return atoms


def _random_real_field(fft, bvec, gcut, sigma, rng):
    """Real grid field sum_G f(G) exp(iG.r) with f ~ CN(0, sigma^2) for 0<|G|<gcut."""
    from .model import grid_miller
    m = grid_miller(fft)
    g = np.linalg.norm(m @ bvec, axis=1)
    sel = (g < gcut) & (g > 0)
    coef = np.zeros(m.shape[0], dtype=np.complex128)
    nsel = int(sel.sum())
    coef[sel] = sigma * (rng.standard_normal(nsel) + 1j * rng.standard_normal(nsel)) / np.sqrt(2)
    # Hermitian symmetry f(-G) = conj f(G): symmetrise
    neg = miller_to_index(-m, fft)
    coef = 0.5 * (coef + coef[neg].conj())
    f = scipy.fft.ifftn(coef.reshape(fft), workers=-1).ravel() * m.shape[0]
    assert np.max(np.abs(f.imag)) < 1e-9 * max(1.0, np.max(np.abs(f.real)))
    return f.real.copy()


def _gaussian_well(fft, lat, bvec, omega, centre, depth, width):
    """Periodic sum of -depth exp(-|r - R - T|^2 / (2 width^2)) over the lattice vectors T
    on the grid, from its Fourier series (every G of the grid)."""
    from .model import grid_miller
    m = grid_miller(fft)
    g = m @ bvec
    g2 = np.sum(g * g, axis=1)
    vg = -depth * (2 * np.pi * width ** 2) ** 1.5 / omega * np.exp(-0.5 * g2 * width ** 2)
    vg = vg * np.exp(-1j * (g @ centre))
    idx = miller_to_index(m, fft)
    arr = np.zeros(int(np.prod(fft)), dtype=np.complex128)
    arr[idx] = vg
    v = scipy.fft.ifftn(arr.reshape(fft)).reshape(-1) * arr.size
    return np.ascontiguousarray(v.real)


def _kpoints(cfg: Config, bvec):
    k1, k2, k3 = cfg.kgrid
    ks = []
    for i in range(k1):
        for j in range(k2):
            for l in range(k3):
                ks.append(np.array([i / k1, j / k2, l / k3]) @ bvec)
    return np.array(ks)


def _density(coeff, miller, npw, fft, omega, wk):
    """n0(r), m0(r) from occupied spinors (X side at k)."""
    nr = int(np.prod(fft))
    n0 = np.zeros(nr)
    m0 = np.zeros((3, nr))
    for k in range(coeff.shape[0]):
        idx = miller_to_index(miller[k, :npw[k]], fft)
        for n in range(coeff.shape[1]):
            psi = np.zeros((2, nr), dtype=np.complex128)
            psi[:, idx] = coeff[k, n, :, :npw[k]]
            psi = scipy.fft.ifftn(psi.reshape(2, *fft), axes=(1, 2, 3), workers=-1).reshape(2, nr) * nr
            psi /= np.sqrt(omega)
            n0 += wk[k] * np.sum(np.abs(psi) ** 2, axis=0)
            for i in range(3):
                m0[i] += wk[k] * np.real(np.einsum("sr,st,tr->r", psi.conj(), PAULI[i], psi))
    return n0, m0


def exchange_field(n0: np.ndarray, m0: np.ndarray) -> np.ndarray:
    """Slater-exchange field of the self-consistent model, b(r) = g(n, |m|) m_hat with
    g = (v_up - v_dn) / 2, v_s = -(6 n_s / pi)^(1/3), n_up/dn = (n +- |m|)/2 floored at
    1e-4; b = 0 where n < 1e-10 or |m| < 1e-12 n (the SCF step of the model, the part
    of the ground-state calculation the paper takes from pw.x)."""
    c6 = (6.0 / np.pi) ** (1.0 / 3.0)
    mabs = np.sqrt(np.sum(m0 * m0, axis=0))
    nu = np.maximum(0.5 * (n0 + mabs), 1e-4)
    nd = np.maximum(0.5 * (n0 - mabs), 1e-4)
    g = 0.5 * (-c6 * nu ** (1.0 / 3.0) + c6 * nd ** (1.0 / 3.0))
    ok = (n0 >= 1e-10) & (mabs >= 1e-12 * n0)
    out = np.zeros_like(m0)
    out[:, ok] = g[ok] * m0[:, ok] / mabs[ok]
    return out


def make_ground_state(name: str, *, seed: int | None = None, collinear: bool = False,
                      kernel_mask: int = 3, device: str | None = None, tol: float = 1e-9,
                      ecut: float | None = None, q_2pi_a=None, nocc: int | None = None,
                      dense_max: int = 2400, log=None, solver: str = "auto",
                      self_consistent: bool = False, b_ext: float = 0.0,
                      scf_tol: float = 1e-11, scf_mix: float = 0.5,
                      scf_iter: int = 400, kgrid=None) -> GroundState:
    """Build the seeded ground-state bundle for config ``name``.

    collinear=True gives the special case of a uniform field along z with no
    spin-orbit coupling ([H, S_z] = 0).  solver="random" skips the
    diagonalisation and fills the occupied states with random orthonormal
    spinors (same shapes; for kernel profiling only, not a ground state).
    kgrid overrides the config's Monkhorst-Pack grid (e.g. a few k points of a large
    cell for tests that need its FFT grid and spheres but not all its k points).
    self_consistent=True replaces the model field by the exchange field of the
    ground state's own magnetisation (exchange_field) plus a uniform external field
    b_ext along z, iterated with linear mixing until the field changes by less than
    scf_tol (dense diagonalisation only).  With spin-orbit coupling off, a uniform
    rotation of the magnetisation then precesses at exactly 2 b_ext (Larmor; zero
    for b_ext = 0, the Goldstone case).
    """
    cfg = dataclasses.replace(CONFIGS[name])
    if seed is not None:
        cfg.seed = seed
    if ecut is not None:
        cfg.ecut = ecut
    if q_2pi_a is not None:
        cfg.q_2pi_a = tuple(q_2pi_a)
    if nocc is not None:
        cfg.nocc = nocc
    if kgrid is not None:
        cfg.kgrid = tuple(kgrid)
    if collinear:
        cfg.b_noncollinear = 0.0
        cfg.lam_so_scale = 0.0
    rng = np.random.default_rng(cfg.seed)
    lat = cfg.lattice
    bvec = reciprocal(lat)
    omega = cell_volume(lat)
    fft = cfg.fft
    nr = int(np.prod(fft))
    vloc = _random_real_field(fft, bvec, cfg.v_gcut, cfg.v_sigma, rng)
    if cfg.b_noncollinear > 0:
        d = np.stack([_random_real_field(fft, bvec, 1.5, 1.0, rng) for _ in range(3)])
        d *= cfg.b_noncollinear / np.sqrt(np.mean(np.sum(d * d, axis=0)))
        d[2] += 1.0
    else:
        d = np.zeros((3, nr))
        d[2] = 1.0
    bfield = cfg.b0 * d / np.linalg.norm(d, axis=0)[None, :]
    atoms = _atoms(cfg, rng)
    for shift in cfg.well_shifts if cfg.well_depth > 0 else ():
        vloc = vloc + _gaussian_well(fft, lat, bvec, omega, atoms[0].tau + np.asarray(shift),
                                     cfg.well_depth, cfg.well_width)
    dnl = block_diag([atom_dmatrix(a) for a in atoms])
    nproj = dnl.shape[0] // 2
    kpts = _kpoints(cfg, bvec)
    nk = kpts.shape[0]
    wk = np.full(nk, 1.0 / nk)
    q = np.array(cfg.q_2pi_a, dtype=np.float64) * 2 * np.pi / cfg.alat
    if self_consistent:
        bfield = _scf_field(cfg, kpts, wk, bvec, omega, fft, vloc, bfield, atoms, dnl, b_ext,
                            scf_tol, scf_mix, scf_iter, dense_max)
    sph_k = [sphere(k, bvec, cfg.ecut, fft) for k in kpts]
    sph_kq = [sphere(k + q, bvec, cfg.ecut, fft) for k in kpts]
    npwx = max(max(s.shape[0] for s in sph_k), max(s.shape[0] for s in sph_kq))
    nb = cfg.nocc
    coeff_k = np.zeros((2, nk, nb, 2, npwx), dtype=np.complex128)
    coeff_kq = np.zeros_like(coeff_k)
    evals = np.zeros((2, nk, nb))
    evals_kq = np.zeros((2, nk, nb))
    gaps = []
    resid_max = 0.0
    beta_kq = np.zeros((nk, nproj, npwx), dtype=np.complex128)
    torch = None
    warm = {}
    for ik, k in enumerate(kpts):
        for which, (p, mil) in enumerate(((k, sph_k[ik]), (k + q, sph_kq[ik]))):
            beta = projector_values(p, mil, bvec, omega, atoms)
            if which == 1:
                beta_kq[ik, :, :mil.shape[0]] = beta
            npw = mil.shape[0]
            for side, sgn in enumerate((+1, -1)):
                if solver == "random":
                    # shape-only bundle for kernel profiling: random orthonormal "occupied"
                    # states and a spread of energies, no diagonalisation
                    a = rng.standard_normal((2 * npw, nb + 1)) + 1j * rng.standard_normal(
                        (2 * npw, nb + 1))
                    v, _ = np.linalg.qr(a)
                    w = np.linspace(-1.0, 0.0, nb + 1)
                    w[nb] = 0.5
                    res = float("nan")
                elif 2 * npw <= dense_max:
                    h = dense_hamiltonian(sgn, p, mil, bvec, fft, vloc, bfield, beta, dnl)
                    w, v = dense_lowest(h, nb + 1)
                    res = np.linalg.norm(h @ v[:, :nb] - v[:, :nb] * w[None, :nb], axis=0).max()
                else:
                    if torch is None:
                        import torch as _torch
                        torch = _torch
                        if device is None:
                            device = "cuda" if torch.cuda.is_available() else "cpu"
                    import time as _time
                    _t0 = _time.time()
                    w, v, res = _iterative(torch, device, sgn, p, mil, bvec, fft, vloc, bfield,
                                           beta, dnl, nb, tol, rng, None, warm.get(side))
                    warm[side] = (mil, v)
                    if log is not None:
                        log(f"  H(k={ik}, {'k+q' if which else 'k'}, side {'XY'[side]}): "
                            f"npw {npw}, resid {res:.1e}, {_time.time() - _t0:.1f} s on {device}")
                resid_max = max(resid_max, float(res))
                gaps.append(float(w[nb] - w[nb - 1]))
                vec = v[:, :nb].T.reshape(nb, 2, npw)
                tgt_c = coeff_k if which == 0 else coeff_kq
                tgt_e = evals if which == 0 else evals_kq
                tgt_c[side, ik, :, :, :npw] = vec
                tgt_e[side, ik] = w[:nb]
    if min(gaps) < 1e-3:
        raise ValueError(f"{name}: gap {min(gaps):.2e} Ha below 1e-3; re-seed")
    miller_k = np.zeros((nk, npwx, 3), dtype=np.int32)
    miller_kq = np.zeros((nk, npwx, 3), dtype=np.int32)
    for ik in range(nk):
        miller_k[ik, :sph_k[ik].shape[0]] = sph_k[ik]
        miller_kq[ik, :sph_kq[ik].shape[0]] = sph_kq[ik]
    n0, m0 = _density(coeff_k[0], miller_k, [s.shape[0] for s in sph_k], fft, omega, wk)
    gs = GroundState(
        lattice=lat, fft=tuple(fft), ecutwfc=float(cfg.ecut), nk=nk, kpts=kpts, q=q, wk=wk,
        nocc=nb, npwx=int(npwx),
        npw_k=np.array([s.shape[0] for s in sph_k], dtype=np.int32),
        npw_kq=np.array([s.shape[0] for s in sph_kq], dtype=np.int32),
        miller_k=miller_k, miller_kq=miller_kq, evals=evals, evals_kq=evals_kq,
        coeff_k=coeff_k, coeff_kq=coeff_kq, vloc=vloc, bfield=bfield, n0=n0, m0=m0,
        nproj=nproj, beta_kq=beta_kq, dnl=dnl, kernel_mask=int(kernel_mask),
        meta={"config": name, "seed": cfg.seed, "gap_min": min(gaps), "resid_max": resid_max,
              "collinear": collinear},
    )
    return gs


def _scf_field(cfg, kpts, wk, bvec, omega, fft, vloc, b_start, atoms, dnl, b_ext, scf_tol, mix,
               niter, dense_max):
    """Fixed point b = exchange_field(n0[b], m0[b]) + b_ext z by linear mixing (X side at k)."""
    nb = cfg.nocc
    b = b_start.copy()
    sph = [sphere(k, bvec, cfg.ecut, fft) for k in kpts]
    betas = [projector_values(k, mil, bvec, omega, atoms) for k, mil in zip(kpts, sph)]
    for it in range(niter):
        coeff = np.zeros((len(kpts), nb, 2, max(m.shape[0] for m in sph)), dtype=np.complex128)
        for ik, (k, mil) in enumerate(zip(kpts, sph)):
            if 2 * mil.shape[0] > dense_max:
                raise ValueError("self-consistent model: dense diagonalisation only")
            h = dense_hamiltonian(+1, k, mil, bvec, fft, vloc, b, betas[ik], dnl)
            w, v = dense_lowest(h, nb + 1)
            coeff[ik, :, :, :mil.shape[0]] = v[:, :nb].T.reshape(nb, 2, mil.shape[0])
        miller = np.zeros((len(kpts), coeff.shape[-1], 3), dtype=np.int32)
        for ik, mil in enumerate(sph):
            miller[ik, :mil.shape[0]] = mil
        n0, m0 = _density(coeff, miller, [m.shape[0] for m in sph], fft, omega, wk)
        b_new = exchange_field(n0, m0)
        b_new[2] += b_ext
        change = float(np.max(np.abs(b_new - b)))
        if change < scf_tol:
            return b_new
        b = (1.0 - mix) * b + mix * b_new
    raise ValueError(f"self-consistent model: no convergence (last change {change:.2e})")


def _iterative(torch, device, sgn, p, mil, bvec, fft, vloc, bfield, beta, dnl, nb, tol, rng, log,
               warm=None):
    """LOBPCG for the lowest nb+1 states; warm = (miller, X) of a neighbouring solve of the
    same side, mapped onto this sphere by Miller index as the starting block."""
    npw = mil.shape[0]
    h = HamiltonianFFT(torch, device, sgn, p, mil, bvec, fft, vloc, bfield, beta, dnl)
    nev = nb + 1
    m = nev + max(4, nev // 5)
    kin = torch.as_tensor(np.concatenate([0.5 * np.sum((p[None, :] + mil @ bvec) ** 2, 1)] * 2),
                          device=device)
    x0 = np.zeros((2 * npw, m), dtype=np.complex128)
    if warm is not None:
        wmil, wx = warm
        key = lambda a: ((a[:, 0].astype(np.int64) + 512) * 1024 + a[:, 1] + 512) * 1024 + a[:, 2] + 512  # noqa: E731
        wk_, nk_ = key(wmil), key(mil)
        order_w = np.argsort(wk_)
        pos = np.searchsorted(wk_[order_w], nk_)
        pos = np.minimum(pos, len(wk_) - 1)
        hit = wk_[order_w][pos] == nk_
        src = order_w[pos[hit]]
        nw_ = wmil.shape[0]
        x0[:npw][hit] = wx[:nw_][src]
        x0[npw:][hit] = wx[nw_:][src]
        x0 += 1e-3 * (rng.standard_normal(x0.shape) + 1j * rng.standard_normal(x0.shape))
    else:
        order = np.argsort(np.concatenate([np.sum((p[None, :] + mil @ bvec) ** 2, 1)] * 2),
                           kind="stable")
        for j in range(m):
            x0[order[j], j] = 1.0
        x0 += 0.05 * (rng.standard_normal(x0.shape) + 1j * rng.standard_normal(x0.shape))
    x0t = torch.as_tensor(x0, device=device)

    def apply_cols(xc):
        xb = xc.T.reshape(-1, 2, npw)
        return h(xb).reshape(xc.shape[1], 2 * npw).T

    theta, x, res = lobpcg(torch, apply_cols, kin, x0t, nev, tol=tol, log=log)
    xn = x.cpu().numpy()
    return theta.cpu().numpy(), xn, float(res[:nb].max())
