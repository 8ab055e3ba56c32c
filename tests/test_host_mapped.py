"""Host-side mapped-domain set-up of the library (quadrature points, stencil
assembly, element stiffness, separation, weighted factors) against the oracle.
CPU only: no device calls."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry, mapped, matrices as omat
from paper_1909_07309_gb300 import stfd

GEOMS = {"box": stfd.STFD_GEOM_BOX, "quarter_annulus": stfd.STFD_GEOM_QUARTER_ANNULUS,
         "revolved_quarter_annulus": stfd.STFD_GEOM_REVOLVED_QUARTER_ANNULUS}


def kappa_lib(x):          # x: (d, m)
    return 1 + 0.5 * np.sin(2 * np.pi * x[0]) * np.cos(2 * np.pi * x[1])


def c_lib(x):
    return 1 + 0.3 * x[0] * x[1]


def kappa_or(x):           # x: (..., d)
    return kappa_lib(np.moveaxis(x, -1, 0))


def c_or(x):
    return c_lib(np.moveaxis(x, -1, 0))


def stencil_to_csr(st, d, p, n_s):
    """Expand the tensor-product stencil layout (as documented in stfd.h) to CSR."""
    W = 2 * p + 1
    Ns = n_s ** d
    rows, cols, vals = [], [], []
    idx = np.arange(Ns)
    multi = [(idx // n_s ** l) % n_s for l in range(d)]
    for o in range(W ** d):
        off = [(o // W ** l) % W - p for l in range(d)]
        ok = np.ones(Ns, dtype=bool)
        j = np.zeros(Ns, dtype=np.int64)
        for l in range(d):
            jl = multi[l] + off[l]
            ok &= (jl >= 0) & (jl < n_s)
            j += np.clip(jl, 0, n_s - 1) * n_s ** l
        assert np.all(st[o][~ok] == 0.0)
        rows.append(idx[ok])
        cols.append(j[ok])
        vals.append(st[o][ok])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(Ns, Ns)).tocsr()


@pytest.mark.parametrize("d,p,n_el,geom,nq", [(2, 3, 5, "quarter_annulus", 4), (2, 2, 6, "box", 3),
                                              (3, 2, 3, "quarter_annulus", 3), (2, 4, 4, "quarter_annulus", 6),
                                              (1, 2, 7, "box", 3), (3, 3, 3, "revolved_quarter_annulus", 4)])
def test_spatial_assembly_matches_oracle(d, p, n_el, geom, nq):
    var = geom != "box"
    xq = stfd.spatial_quadrature_points(d, p, n_el, GEOMS[geom], nq)
    Ms, Ks = stfd.spatial_assemble(d, p, n_el, GEOMS[geom], nq, c_lib(xq) if var else None,
                                   kappa_lib(xq) if var else None)
    oMs, oKs = mapped.spatial_matrices(d, p, n_el, geom, c=c_or if var else None, kappa=kappa_or if var else None,
                                       nq=nq)
    n_s = n_el + p - 2
    for st, ref in ((Ms, oMs), (Ks, oKs)):
        A = stencil_to_csr(st, d, p, n_s)
        assert abs(A - ref).max() <= 1e-14 * abs(ref).max()


def test_quadrature_points_are_the_mapped_gauss_points():
    d, p, n_el, nq = 2, 2, 3, 3
    x = stfd.spatial_quadrature_points(d, p, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS, nq)
    t, _ = np.polynomial.legendre.leggauss(nq)
    k = 0
    for e2 in range(n_el):
        for e1 in range(n_el):
            for q2 in range(nq):
                for q1 in range(nq):
                    eta = np.array([(e1 + 0.5 * (t[q1] + 1)) / n_el, (e2 + 0.5 * (t[q2] + 1)) / n_el])
                    ref, _ = geometry.quarter_annulus(eta[None, :])
                    assert np.max(np.abs(x[:, k] - ref[0])) <= 1e-15
                    k += 1


def test_element_stiffness_sums_to_piecewise_constant_conductivity():
    d, p, n_el, nq = 2, 3, 4, 4
    g = np.random.default_rng(1)
    kap = g.uniform(0.5, 2.0, n_el ** d)
    Ke = stfd.spatial_element_stiffness(d, p, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS, nq)
    _, oKs, elems = mapped.spatial_matrices(d, p, n_el, kappa_elem=kap, nq=nq, element_stiffness=True)
    n_s = n_el + p - 2
    K = np.zeros((n_s ** d, n_s ** d))
    L = p + 1
    for e in range(n_el ** d):
        e1, e2 = e % n_el, e // n_el
        rows = []
        for a in range(L ** d):
            i1, i2 = e1 + a % L - 1, e2 + a // L - 1
            rows.append(i1 + n_s * i2 if (0 <= i1 < n_s and 0 <= i2 < n_s) else -1)
        rows = np.array(rows)
        ok = rows >= 0
        K[np.ix_(rows[ok], rows[ok])] += kap[e] * Ke[e][np.ix_(ok, ok)]
        gi, Ko = elems[e]
        assert np.max(np.abs(Ke[e][np.ix_(ok, ok)] - Ko)) <= 1e-14 * np.max(np.abs(Ko))
    assert np.max(np.abs(K - oKs.toarray())) <= 1e-14 * abs(oKs).max()
    # the stencil assembly with the same piecewise-constant conductivity agrees
    _, Ks = stfd.spatial_assemble(d, p, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS, nq, None, np.repeat(kap, nq ** d))
    assert abs(stencil_to_csr(Ks, d, p, n_s) - oKs).max() <= 1e-14 * abs(oKs).max()


@pytest.mark.parametrize("d,n_el", [(2, 6), (3, 4)])
def test_separation_matches_oracle(d, n_el):
    xm = stfd.spatial_element_midpoints(d, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS)
    phi, Phi = stfd.geo_separate(d, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS, c_lib(xm), kappa_lib(xm))
    Cd = mapped.coefficient_diagonal(d, n_el, "quarter_annulus", c=c_or, kappa=kappa_or)
    ophi, oPhi = mapped.separate(Cd, d, n_el)
    assert np.max(np.abs(phi - ophi) / ophi) <= 1e-13 and np.max(np.abs(Phi - oPhi) / oPhi) <= 1e-13


def test_weighted_univariate_matrices_match_oracle():
    p, n_el = 3, 7
    g = np.random.default_rng(2)
    wm, ws = g.uniform(0.5, 2, n_el), g.uniform(0.5, 2, n_el)
    M, K = stfd.spline_matrices_weighted(p, n_el, 1.0, stfd.STFD_BC_DIRICHLET, wm, ws)
    oK, oM = mapped.weighted_matrices(p, n_el, wm, ws)
    assert np.max(np.abs(M - oM)) <= 1e-15 and np.max(np.abs(K - oK)) <= 1e-12
    # unit weights reduce to the unweighted factors
    M1, K1 = stfd.spline_matrices_weighted(p, n_el, 1.0, stfd.STFD_BC_DIRICHLET)
    K0, M0 = omat.space_matrices(p, n_el)
    assert np.max(np.abs(M1 - M0)) <= 1e-15 and np.max(np.abs(K1 - K0)) <= 1e-12


def test_mapped_api_rejects_bad_arguments():
    lib = stfd.load()
    x = np.zeros(100)
    assert lib.stfd_spatial_quadrature_points(1, 2, 3, stfd.STFD_GEOM_QUARTER_ANNULUS, 3, stfd._dptr(x)) == -1
    assert lib.stfd_spatial_assemble(2, 2, 3, 7, 3, None, None, stfd._dptr(x), None) == -1
    assert lib.stfd_geo_separate(2, 3, stfd.STFD_GEOM_BOX, None, None, None, None) == -1
    bad = -np.ones(9)
    phi = np.zeros(6)
    assert lib.stfd_geo_separate(2, 3, stfd.STFD_GEOM_BOX, None, stfd._dptr(bad), stfd._dptr(phi),
                                 stfd._dptr(phi)) == -1
