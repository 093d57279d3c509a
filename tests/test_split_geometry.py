"""The single enclosing domain against two sub-domains (Sec. III, Eq. 13).

The comparison times one domain of d' x W' x L' nodes holding both
sub-domains' sources (zeros in the gap) against the two W' x W' x L'
sub-domains themselves.  Both must give the same potentials at the
sub-domains' nodes, since the gap's nodes carry no source.  These CPU checks
pin the geometry helpers and that identity on the FP64 oracle.
"""
import numpy as np

import oracle
from paper_2311_15429_gb300 import synth


def test_embedding_places_each_subdomain_at_its_own_nodes():
    g = synth.split_geometry(4, 6, 11, 0.25)
    x, y, z = g.enclosing.coords()
    for k in range(2):
        xs, ys, zs = g.subs[k].coords()
        n = g.sub_nodes(k)
        assert np.allclose(x[n], xs) and np.allclose(y[n], ys) and np.allclose(z[n], zs)
    hist = [s.history(0, 3, 0.05) for s in g.sources]
    e = g.embed(hist)
    gap = np.ones(g.enclosing.N, bool)
    for k in range(2):
        assert np.array_equal(e[:, :, g.sub_nodes(k)], hist[k])
        gap[g.sub_nodes(k)] = False
    assert gap.sum() == g.enclosing.N - 2 * g.subs[0].N
    assert np.all(e[:, :, gap] == 0)


def test_enclosing_domain_equals_two_subdomains_on_the_oracle():
    """Retarded sums at sub-domain nodes: one enclosing domain with zero gap
    sources against the two sub-domains (several lags, both the self cell
    and cross terms)."""
    g = synth.split_geometry(3, 5, 9, 0.4)
    c, dt, T = synth.C_AU, 0.004, 12
    hist = [s.history(0, T, dt) for s in g.sources]
    big = [g.embed(hist)]
    step = T - 1
    for k in range(2):
        nodes = np.arange(g.subs[k].N)
        two = oracle.eval_points([d.origin for d in g.subs], [d.n for d in g.subs], [d.h for d in g.subs],
                                 hist, 0, c, dt, k, step, nodes)
        one = oracle.eval_points([g.enclosing.origin], [g.enclosing.n], [g.enclosing.h], big, 0, c, dt, 0,
                                 step, g.sub_nodes(k))
        np.testing.assert_allclose(one, two, rtol=1e-13, atol=1e-13 * np.abs(two).max())
