"""Pins of the variable-fixing oracle (oracle/fix.py, Sec. 6.1).

* A worked example derived by hand: a 5x3x3 mesh whose elements ex >= 2
  are void and ex <= 1 solid.  Void: ex = 2, 3, 4.  Fixed void: ex = 3, 4
  (every neighbour of ex = 3 is in ex = 2..4; ex = 4 has no neighbour
  beyond the domain).  Solid: ex = 0, 1; fixed solid: ex = 0 only (ex = 1
  touches ex = 2).  Suppressed nodes: those whose every element is in
  ex = 3, 4, i.e. lattice columns i = 4, 5 for degree 1 (i = 3 touches
  ex = 2) and i = 7..10 for degree 2 (i = 6 is shared with ex = 2).
* The gradient safeguards: one design variable with a gradient below
  -eps_grad keeps its element from being void.
* The fixed set against a library routine (a 3x3x3 minimum filter), the
  suppressed nodes against the element-node incidence of the assembly.
* The physics the section relies on: with Emin = 1e-9 E0, suppressing the
  nodes of a fixed void region changes the compliance by a relative amount
  of order Emin (pinned at 1e-6), while suppressing one layer more (the
  nodes on the border of the structure) changes it by orders of magnitude
  more.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

import workloads
from oracle import fe, fix, mesh


def _block_problem(k, n=2, shape=(5, 3, 3), void_from=2):
    p = workloads.cantilever(*shape, degree=k, n_mr=n, seed=0)
    Dx = n * shape[0]
    cx = np.arange(p.x.size) % Dx
    p.x = np.where(cx >= n * void_from, 0.0, 1.0)
    return p


@pytest.mark.parametrize("k,cols", [(1, [4, 5]), (2, [7, 8, 9, 10])])
def test_worked_example(k, cols):
    p = _block_problem(k)
    cls = fix.element_class(p, p.x, None, 1e-6, 0.9, 1e-6)
    ex = np.arange(cls.size) % 5
    assert np.array_equal(cls, np.where(ex >= 2, fix.VOID, fix.SOLID))
    fx = fix.fixed_elements(p, cls)
    want = np.select([ex >= 3, ex == 0], [fix.VOID, fix.SOLID], 0)
    assert np.array_equal(fx, want)
    sup = fix.suppressed_nodes(p, fx)
    Lx, Ly, Lz = p.lattice
    i = np.arange(sup.size) % Lx
    assert np.array_equal(sup, np.isin(i, cols))
    assert sup.sum() == len(cols) * Ly * Lz
    fxv = fix.fixed_design_variables(p, fx)
    cx = np.arange(p.x.size) % 10
    assert np.array_equal(fxv, np.select([cx >= 6, cx <= 1], [fix.VOID, fix.SOLID], 0))


def test_gradient_safeguards():
    p = _block_problem(1)
    g = np.zeros(p.x.size)
    cell = 9 + 10 * (1 + 6 * 2)  # cx = 9 (element ex = 4), cy = 1, cz = 2
    g[cell] = -1e-3
    cls = fix.element_class(p, p.x, g, 1e-6, 0.9, 1e-6)
    assert cls.reshape(3, 3, 5)[1, 0, 4] == 0
    fx = fix.fixed_elements(p, cls)
    assert fx.reshape(3, 3, 5)[1, 0, 3] == 0  # its neighbour is no longer fixed
    g2 = np.zeros(p.x.size)
    g2[0] = 1e-3  # a solid element whose variable would decrease
    cls2 = fix.element_class(p, p.x, g2, 1e-6, 0.9, 1e-6)
    assert cls2[0] == 0 and cls2[1] == fix.SOLID
    # within the tolerance nothing changes
    cls3 = fix.element_class(p, p.x, np.full(p.x.size, 0.5e-6), 1e-6, 0.9, 1e-6)
    assert np.array_equal(cls3, fix.element_class(p, p.x, None, 1e-6, 0.9, 1e-6))


def test_all_void_and_nothing_void():
    p = workloads.cantilever(4, 3, 2, degree=2, n_mr=1, seed=0)
    cls = fix.element_class(p, np.zeros(p.x.size), None, 1e-6, 0.9, 1e-6)
    fx = fix.fixed_elements(p, cls)
    assert (fx == fix.VOID).all() and fix.suppressed_nodes(p, fx).all()
    cls = fix.element_class(p, np.full(p.x.size, 0.5), None, 1e-6, 0.9, 1e-6)
    fx = fix.fixed_elements(p, cls)
    assert (fx == 0).all() and not fix.suppressed_nodes(p, fx).any()


@pytest.mark.parametrize("k,shape", [(1, (7, 5, 4)), (2, (5, 4, 3))])
def test_fixed_set_and_nodes_against_independent_constructions(k, shape):
    p = workloads.cantilever(*shape, degree=k, n_mr=2, seed=4)
    rng = np.random.default_rng(1)
    ev = rng.random(shape[0] * shape[1] * shape[2]) < 0.8  # void elements
    rho = np.ones(p.x.size)
    rho[mesh.subcell_density_index(*shape, 2)[ev].reshape(-1)] = 0.0
    cls = fix.element_class(p, rho, None, 1e-6, 0.9, 1e-6)
    assert np.array_equal(cls == fix.VOID, ev)
    fx = fix.fixed_elements(p, cls)
    v3 = ev.reshape(shape[2], shape[1], shape[0]).astype(np.uint8)
    want = ndi.minimum_filter(v3, size=3, mode="constant", cval=1).reshape(-1).astype(bool) & ev
    assert np.array_equal(fx == fix.VOID, want)
    # a node is kept iff some element containing it is not fixed void
    kept = np.zeros(p.nnodes, dtype=bool)
    ed = mesh.element_dofs(*shape, k)
    kept[ed[fx != fix.VOID][:, 0::3].reshape(-1) // 3] = True
    assert np.array_equal(fix.suppressed_nodes(p, fx), ~kept)


def test_gradient_components_of_fixed_void_variables_are_zero():
    g = np.array([-1.0, -2.0, -3.0, -4.0])
    out = fix.zero_fixed_void_gradient(g, np.array([0, 1, 2, 1], dtype=np.int8))
    assert np.array_equal(out, [-1.0, 0.0, -3.0, 0.0])


@pytest.mark.parametrize("k", [1, 2])
def test_suppression_changes_compliance_by_order_emin(k):
    """Cantilever solid in its bottom half (ez < 2), void above, loaded at
    the bottom edge: the fixed void layer is ez = 3, and the nodes above its
    lower face (l > 3k) are suppressed."""
    shape = (8, 4, 4)
    p = workloads.cantilever(*shape, degree=k, n_mr=1, seed=0)
    cz = np.arange(p.x.size) // (shape[0] * shape[1])
    p.x = np.where(cz < 2, 1.0, 0.0)
    cls = fix.element_class(p, p.x, None, 1e-6, 0.9, 1e-6)
    fx = fix.fixed_elements(p, cls)
    assert np.array_equal(fx == fix.VOID, cz == 3)
    sup = fix.suppressed_nodes(p, fx)
    Lx, Ly, Lz = p.lattice
    l = np.arange(p.nnodes) // (Lx * Ly)
    assert np.array_equal(sup, l > 3 * k)  # l = 3k is shared with ez = 2
    c_full = fe.Model(p).run(method="splu")["c"][0]
    q = fix.suppressed_problem(p, sup)
    c_sup = fe.Model(q).run(method="splu")["c"][0]
    assert abs(c_sup - c_full) <= 1e-6 * c_full
    # one layer more (down to the top face of the structure) is not negligible
    q2 = fix.suppressed_problem(p, l >= 2 * k)
    c_bad = fe.Model(q2).run(method="splu")["c"][0]
    assert abs(c_bad - c_full) > 1e-3 * c_full
