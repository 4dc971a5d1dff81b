"""The seeded synthetic workloads against their stated recipe (CPU).

The generators stand in for the paper's thermo-structure interaction (Sec.
6.1) and coupled 3D systems: Q1 elasticity (plane strain in 2D), transient heat
k*L + M/dt, a scalar diffusion field with a per-cell diffusivity, coupling
blocks A_01 = alpha * int B^T m N and A_10 = beta * int N m^T B (so A_10 =
(beta/alpha) A_01^T), the x = 0 boundary clamped by symmetric elimination.
Checked from the mathematics, not by re-running the assembly: dof counts,
symmetry, the coupling ratio, rigid-body modes in the kernel of the elasticity
rows away from the boundary, constants in the kernel of the Laplacians, the
Q1 mass row sum h^d, identity rows and zero couplings on the boundary, the
log-uniform batch sizes, and the structure of the split-box saddle system."""
import numpy as np
import pytest

from paper_1605_01522_gb300 import inputs


def _blocks(s):
    return s.scipy_blocks()


def _interior_rows(f, ne, dim, margin=2):
    """Nodes at least `margin` cells away from the clamped x = 0 face (their
    rows touch no eliminated column), as dof indices of field f."""
    x = np.rint(f.coords[:, 0] * ne).astype(int)
    nodes = np.nonzero(x >= margin)[0]
    return (nodes[:, None] * f.b + np.arange(f.b)[None, :]).ravel()


def _rbm(coords, dim):
    """Rigid-body modes of a displacement field: translations and rotations."""
    n = coords.shape[0]
    modes = []
    for d in range(dim):
        m = np.zeros((n, dim))
        m[:, d] = 1.0
        modes.append(m.ravel())
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (0, 2)]
    for a, b in pairs:
        m = np.zeros((n, dim))
        m[:, a] = -coords[:, b]
        m[:, b] = coords[:, a]
        modes.append(m.ravel())
    return modes


def test_thermo_elastic_2d_sizes_symmetry_and_coupling_ratio():
    s = inputs.thermo_elastic_2d(ne=32)
    assert [f.ndofs for f in s.fields] == [2178, 1089] and s.ndofs == 3267
    A = _blocks(s)
    for i in (0, 1):
        d = A[(i, i)]
        assert abs(d - d.T).max() <= 1e-14 * abs(d).max()
    a01, a10 = A[(0, 1)], A[(1, 0)]
    assert abs(a10 - (1e-3 / 1e-2) * a01.T).max() <= 1e-15 * abs(a10).max()
    assert abs(a01).max() > 0


@pytest.mark.parametrize("maker,dim,ne", [(lambda: inputs.thermo_elastic_2d(ne=16), 2, 16),
                                          (lambda: inputs.coupled_box_3d(ne=6, nfields=3), 3, 6)])
def test_elasticity_rows_annihilate_rigid_body_modes_and_laplacians_constants(maker, dim, ne):
    s = maker()
    A = _blocks(s)
    f0 = s.fields[0]
    rows = _interior_rows(f0, ne, dim)
    K = A[(0, 0)]
    for r in _rbm(f0.coords, dim):
        assert abs(K @ r)[rows].max() <= 1e-12 * abs(K).max() * abs(r).max()
    # heat: k*L + M/dt, so the row sums away from the boundary are the Q1
    # mass row sums h^dim over dt (dt = 0.1)
    h = 1.0 / ne
    heat_rows = _interior_rows(s.fields[1], ne, dim)
    rs = np.asarray(A[(1, 1)].sum(axis=1)).ravel()
    interior = heat_rows[np.all((s.fields[1].coords[heat_rows] * ne > 0.5) &
                                (s.fields[1].coords[heat_rows] * ne < ne - 0.5), axis=1)]
    assert np.allclose(rs[interior], h ** dim / 0.1, rtol=1e-12)
    if s.nfields == 3:  # diffusion: a Laplacian with a cell diffusivity, no mass
        rs2 = np.asarray(A[(2, 2)].sum(axis=1)).ravel()
        assert abs(rs2[heat_rows]).max() <= 1e-12 * abs(A[(2, 2)]).max()
        diag = A[(2, 2)].diagonal()[heat_rows]
        assert diag.max() / diag.min() > 10.0  # diffusivity spread over orders of magnitude


def test_clamped_face_identity_rows_zero_couplings_zero_rhs():
    s = inputs.coupled_box_3d(ne=5, nfields=3)
    A = _blocks(s)
    off = s.offsets
    dn = s.fields[0].dirichlet_nodes
    assert len(dn) == 36 and np.all(s.fields[0].coords[dn, 0] == 0.0)
    for i, fi in enumerate(s.fields):
        d = (dn[:, None] * fi.b + np.arange(fi.b)[None, :]).ravel()
        assert np.all(s.rhs[off[i] + d] == 0.0)
        for j, fj in enumerate(s.fields):
            if (i, j) not in A:
                continue
            rows = A[(i, j)].tocsr()[d].toarray()
            if i == j:
                assert np.array_equal(rows[:, d], np.eye(len(d)))
                rows[:, d] = 0.0
            assert not rows.any()
            dj = (dn[:, None] * fj.b + np.arange(fj.b)[None, :]).ravel()
            cols = A[(i, j)].tocsc()[:, dj].toarray()
            if i == j:
                cols[d, :] = 0.0
            assert not cols.any()


def test_batch_sizes_are_log_uniform_in_range():
    sizes = inputs.batch_sizes_log_uniform(4096, 12, 48, seed=3)
    assert sizes.min() >= 12 and sizes.max() <= 48
    # log-uniform: the median sits near the geometric mean sqrt(12 * 48) = 24
    assert abs(np.median(sizes) - 24) <= 1.5
    assert abs(np.mean(np.log(sizes)) - np.log(24)) < 0.03
    s256, mats, rhs = inputs.batch_workload(8, 12, 16, seed=3)
    assert len(rhs) == 8 and all(len(r) == mats[int(n)].ndofs for r, n in zip(rhs, s256))
    assert all(mats[int(n)].fields[0].nnodes == (n + 1) ** 3 for n in s256)


def test_split_box_saddle_system_structure():
    """The split-box saddle stand-in: four fields on the two halves of the cube
    (structure above z = 0.5; mesh motion, Stokes velocity and PSPG pressure
    below), 600,250 dofs at n_e = 48 by the node counts, a symmetric
    gradient / divergence pair, a negative semi-definite stabilised pressure
    block on the free dofs, an S-Fu interface penalty pair, and a symmetric
    velocity block that becomes non-symmetric (and Petrov-Galerkin) with wind."""
    ne = 8
    s = inputs.fsi_box(ne=ne)
    up, lo = (ne + 1) ** 2 * (ne - ne // 2 + 1), (ne + 1) ** 2 * (ne // 2 + 1)
    assert [f.ndofs for f in s.fields] == [3 * up, 3 * lo, 3 * lo, lo]
    assert 3 * 49 ** 2 * 25 * 3 + 49 ** 2 * 25 == 600250  # the n_e = 48 form
    A = _blocks(s)
    assert abs(A[(3, 2)] - A[(2, 3)].T).max() == 0.0
    assert abs(A[(0, 2)] - A[(2, 0)].T).max() == 0.0 and abs(A[(0, 2)]).max() > 0
    assert not any(k in A for k in [(0, 1), (1, 0), (0, 3), (3, 0), (1, 3), (3, 1)])
    fu = A[(2, 2)]
    assert abs(fu - fu.T).max() <= 1e-14 * abs(fu).max()
    fp = s.fields[3]
    free = np.setdiff1d(np.arange(fp.ndofs), fp.dirichlet_nodes)
    P = A[(3, 3)].toarray()[np.ix_(free, free)]
    assert np.linalg.eigvalsh(P).max() <= 1e-12 * abs(P).max()
    assert np.all(np.diag(P) < 0)
    assert not s.fields[2].petrov_galerkin
    o = inputs.fsi_box(ne=ne, wind=(0.2, 0.1, 0.0))
    fo = _blocks(o)[(2, 2)]
    assert abs(fo - fo.T).max() > 1e-6 * abs(fo).max() and o.fields[2].petrov_galerkin
