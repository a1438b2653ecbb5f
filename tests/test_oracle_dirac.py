"""Pins of the oracle's Wilson-clover operator against what the mathematics fixes."""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np
import torch

import synthetic as syn
from oracle.dirac import (GAMMA, GAMMA5, WilsonClover, chiral_blocks,
                          clover_term, gauge_transform, pack_hermitian,
                          unpack_hermitian)
from oracle.lattice import Blocking, Geometry, index_maps
from tests.oracle_fixtures import C128, colour_rotate, dense_D, dot, rel, spinors, t, wilson

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gamma_algebra():
    I4 = torch.eye(4, dtype=C128)
    for a in range(4):
        assert torch.allclose(GAMMA[a], GAMMA[a].conj().T)
        for b in range(4):
            ac = GAMMA[a] @ GAMMA[b] + GAMMA[b] @ GAMMA[a]
            assert torch.allclose(ac, 2.0 * (a == b) * I4)
    assert torch.allclose(GAMMA5, torch.diag(torch.tensor([1, 1, -1, -1], dtype=C128)))


def test_index_maps_bruteforce():
    L = (4, 6, 2, 8)
    g = Geometry(L)
    # lexicographic bijection and neighbours
    seen = set()
    for site in range(g.V):
        x, y, z, tt = (int(v) for v in g.coords[site])
        assert site == x + L[0] * (y + L[1] * (z + L[2] * tt))
        seen.add(site)
        assert int(g.parity[site]) == (x + y + z + tt) % 2
        for mu in range(4):
            c = [x, y, z, tt]
            c[mu] = (c[mu] + 1) % L[mu]
            assert int(g.fwd[mu, site]) == c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))
            # parity alternates along every axis with even extent
            assert int(g.parity[g.fwd[mu, site]]) != int(g.parity[site])
            assert int(g.bwd[mu, g.fwd[mu, site]]) == site
    assert len(seen) == g.V
    b = Blocking(g, (2, 2, 2, 4))
    assert b.n_blocks == 2 * 3 * 1 * 2
    flat = sorted(int(s) for s in b.sites.reshape(-1))
    assert flat == list(range(g.V))
    for B in range(b.n_blocks):
        cs = g.coords[b.sites[B]]
        span = cs.max(0).values - cs.min(0).values + 1
        assert tuple(int(v) for v in span) == (2, 2, 2, 4)
    # colours alternate between neighbouring blocks
    for B in range(b.n_blocks):
        for mu in range(4):
            if b.grid[mu] > 1 and b.grid[mu] % 2 == 0:
                assert int(b.colour_of_block[b.coarse.fwd[mu, B]]) != int(b.colour_of_block[B])


def test_paper_aggregation_example():
    """Sec. 4: a 12x12x12x24 local lattice with 4^4 domains becomes 3x3x3x6,
    and 16 test vectors give 32 degrees of freedom per coarse site."""
    with open(os.path.join(GOLDEN, "paper_facts.json")) as f:
        facts = json.load(f)["aggregation"]
    g = Geometry(facts["fine_lattice"])
    a = Blocking(g, facts["block"])
    assert list(a.grid) == facts["coarse_lattice"]
    assert a.block_volume == 256
    assert 2 * facts["n_v"] == facts["coarse_dof_per_site"]
    assert 12 == facts["fine_dof_per_site"]
    maps = index_maps(facts["fine_lattice"], facts["block"], facts["block"])
    counts = torch.bincount(maps["aggregate"].long())
    assert len(counts) == 3 * 3 * 3 * 6 and bool((counts == 256).all())


def test_gamma5_hermiticity_dense():
    D = dense_D()
    g5 = torch.diag(GAMMA5).real
    s = g5.repeat_interleave(3).repeat(256)
    lhs = s[:, None] * D * s[None, :]
    assert rel(lhs, D.conj().T) < 1e-14


def test_gamma5_hermiticity_random():
    L = (4, 4, 4, 6)
    op = wilson(L, 0.3, 3, -0.1, 1.3)
    phi, psi = spinors(2, L, 11)
    g5 = torch.diag(GAMMA5).real[:, None]
    lhs = dot(phi, g5 * op.apply(g5 * psi))
    rhs = dot(op.apply(phi), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)


def _free_eigen(p, m0):
    re = m0 + sum(1 - math.cos(v) for v in p)
    im = math.sqrt(sum(math.sin(v) ** 2 for v in p))
    return complex(re, im), complex(re, -im)


def test_free_field_plane_waves():
    L = (4, 4, 2, 6)
    m0 = 0.13
    op = WilsonClover(t(syn.unit_gauge(L)), L, m0, 1.7)
    assert float(op.A.sub(torch.eye(12, dtype=C128) * (4 + m0)).abs().max()) == 0.0  # C = 0 on U = 1
    g = op.geom
    rng = np.random.default_rng(5)
    for n in [(1, 0, 1, 2), (0, 3, 0, 5), (2, 1, 1, 0)]:
        p = [2 * math.pi * n[k] / L[k] for k in range(3)] + [(2 * n[3] + 1) * math.pi / L[3]]
        phase = torch.exp(1j * (g.coords.to(torch.float64) @ torch.tensor(p, dtype=torch.float64)))
        u = t(rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3)))
        psi = phase[:, None, None] * u
        Dpsi = op.apply(psi)
        M = (m0 + sum(1 - math.cos(v) for v in p)) * torch.eye(4, dtype=C128)
        for mu in range(4):
            M = M + 1j * math.sin(p[mu]) * GAMMA[mu]
        assert rel(Dpsi, phase[:, None, None] * (M @ u)) < 1e-13


def test_free_field_spectrum_dense():
    L = (2, 2, 4, 4)
    m0 = -0.3
    op = WilsonClover(t(syn.unit_gauge(L)), L, m0, 1.0)
    ev = torch.linalg.eigvals(op.dense()).numpy()
    expect = []
    for n in itertools.product(*(range(v) for v in L)):
        p = [2 * math.pi * n[k] / L[k] for k in range(3)] + [(2 * n[3] + 1) * math.pi / L[3]]
        for lam in _free_eigen(p, m0):
            expect += [lam] * 6
    expect = np.array(expect)
    assert len(ev) == len(expect)
    # greedy nearest matching of the two multisets
    used = np.zeros(len(expect), bool)
    worst = 0.0
    for lam in ev:
        d = np.abs(expect - lam)
        d[used] = np.inf
        k = int(np.argmin(d))
        used[k] = True
        worst = max(worst, d[k])
    assert worst < 1e-12


def test_gauge_covariance():
    L = (4, 4, 4, 6)
    op = wilson(L, 0.3, 3, -0.1, 1.3)
    Om = t(syn.random_su3((op.geom.V,), 1.0, syn.rng(77)))
    Ug = gauge_transform(op.U, Om, op.geom)
    opg = WilsonClover(Ug, L, op.m0, op.csw)
    psi = spinors(1, L, 12)[0]
    lhs = opg.apply(colour_rotate(psi, Om))
    rhs = colour_rotate(op.apply(psi), Om)
    assert rel(lhs, rhs) < 1e-13
    # the clover term itself transforms covariantly
    C = clover_term(op.U, op.geom, op.csw).reshape(-1, 4, 3, 4, 3)
    Cg = clover_term(Ug, op.geom, op.csw).reshape(-1, 4, 3, 4, 3)
    rot = torch.einsum("xab,xsbtc,xdc->xsatd", Om, C, Om.conj())
    assert rel(Cg, rot) < 1e-13


def test_clover_structure():
    op = wilson((4, 4, 4, 6), 0.3, 3, -0.1, 1.3)
    C = op.A - (4 + op.m0) * torch.eye(12, dtype=C128)
    assert float(C.abs().max()) > 1e-2
    assert rel(C, C.conj().transpose(-1, -2)) < 1e-15          # Hermitian
    assert float(C[:, 0:6, 6:12].abs().max()) < 1e-15             # commutes with g5
    assert float(C[:, 6:12, 0:6].abs().max()) < 1e-15


def test_clover_constant_abelian_field():
    """Constant U(1) flux phi per x-y plaquette embedded along T = diag(1,1,-2):
    every leaf is exp(i phi T), so F_xy = sin(phi T) and
    C = -(i csw / 2) g_x g_y (x) sin(phi T); all other planes vanish."""
    L = (4, 6, 2, 2)
    g = Geometry(L)
    T = torch.tensor([1.0, 1.0, -2.0], dtype=torch.float64)
    phi = 2 * math.pi * 1 / (L[0] * L[1])
    U = torch.zeros((g.V, 4, 3, 3), dtype=C128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1.0
    x, y = g.coords[:, 0].double(), g.coords[:, 1].double()
    U[:, 1] = torch.diag_embed(torch.exp(1j * phi * x[:, None] * T))
    edge = g.coords[:, 0] == L[0] - 1
    U[edge, 0] = torch.diag_embed(torch.exp(-1j * phi * L[0] * y[edge][:, None] * T))
    csw = 1.37
    C = clover_term(U, g, csw)
    expect = -(1j * csw / 2) * torch.kron(GAMMA[0] @ GAMMA[1],
                                          torch.diag(torch.sin(phi * T)).to(C128))
    assert rel(C, expect.expand(g.V, 12, 12)) < 1e-14


def test_clover_inverse_and_packing():
    op = wilson((4, 4, 4, 6), 0.3, 3, -0.1, 1.3)
    I = torch.eye(12, dtype=C128).expand(op.geom.V, 12, 12)
    assert rel(op.A @ op.Ainv, I) < 1e-14
    P = op.packed_clover()
    assert P.shape == (op.geom.V, 2, 36)                          # 6 real + 15 complex
    B = chiral_blocks(op.A)
    assert rel(unpack_hermitian(P), B) < 1e-16
    assert rel(pack_hermitian(unpack_hermitian(P)), P) == 0.0
    Pi = op.packed_clover(inverse=True)
    assert rel(unpack_hermitian(Pi) @ B, torch.eye(6, dtype=C128).expand_as(B)) < 1e-14


def test_antiperiodic_time_boundary():
    """With antiperiodic t the unit-link operator has no p_t = 0 mode: the
    smallest |eigenvalue| of the free operator at m0 = 0 is nonzero, while the
    periodic operator has an exact zero mode."""
    L = (2, 2, 2, 4)
    ap = WilsonClover(t(syn.unit_gauge(L)), L, 0.0, 1.0).dense()
    per = WilsonClover(t(syn.unit_gauge(L)), L, 0.0, 1.0, antiperiodic_t=False).dense()
    assert torch.linalg.eigvals(per).abs().min().item() < 1e-12
    assert torch.linalg.eigvals(ap).abs().min().item() > 0.5
