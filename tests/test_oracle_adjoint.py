"""Pins for the oracle's adjoints: the marching-cubes position adjoint and the
distance-to-original-surface loss, both checked against central finite
differences of the oracle's own float64 forward, plus closed forms."""
import numpy as np

import oracle
from paper_2408_05462_gb300 import synth


def _safe_vertices(f, k, h, n, seed):
    """Vertices whose every incident crossing edge is well away from
    degenerate (|f1 - f0| > 1e-2) and whose value is further than 2h from k,
    so a +-h step changes no case."""
    nz, ny, nx = f.shape
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    tries = 0
    while len(out) < n and tries < 100000:
        tries += 1
        z, y, x = (int(g.integers(1, s - 1)) for s in (nz, ny, nx))
        v = f[z, y, x]
        if abs(v - k) <= 2 * h:
            continue
        ok, crossing = True, False
        for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            w = f[z + dz, y + dy, x + dx]
            if (v < k) != (w < k):
                crossing = True
                if abs(w - v) <= 1e-2:
                    ok = False
        if ok and crossing:
            out.append((z, y, x))
    return out


def test_mc_backward_matches_finite_differences():
    f = synth.turbulence(20, seed=5)
    k = 0.2
    m = oracle.mc(f, k)
    G = np.random.Generator(np.random.PCG64(1)).normal(size=m.pos.shape)
    grad = oracle.mc_backward(f, k, G)
    h = 1e-5
    for (z, y, x) in _safe_vertices(f, k, h, 25, 2):
        fp, fm = f.copy(), f.copy()
        fp[z, y, x] += np.float32(h)
        fm[z, y, x] -= np.float32(h)
        mp, mm = oracle.mc(fp, k), oracle.mc(fm, k)
        assert mp.ntri == mm.ntri == m.ntri
        fd = (np.sum(G * mp.pos) - np.sum(G * mm.pos)) / (float(fp[z, y, x]) - float(fm[z, y, x]))
        assert abs(fd - grad[z, y, x]) <= 1e-5 * max(1.0, abs(fd)), (z, y, x, fd, grad[z, y, x])


def test_mc_backward_of_a_plane():
    # f = z - c: the surface is z = c, and moving f at the two ends of a
    # z-edge moves the vertex by (t-1)/(f1-f0) and -t/(f1-f0) with f1-f0 = 1
    nx, ny, nz = 6, 5, 7
    f = synth.plane_field((nx, ny, nz), (0, 0, 1), 3.25)
    m = oracle.mc(f, 0.0)
    G = np.zeros_like(m.pos)
    G[:, :, 2] = 1.0  # L = sum of all vertex z coordinates
    grad = oracle.mc_backward(f, 0.0, G)
    t = 0.25
    # every z-edge between z = 3 and z = 4 carries the uses of its vertex
    uses = np.zeros((ny, nx))
    for tri in m.edge_id:
        for eid in tri:
            i0, axis = divmod(int(eid), 3)
            assert axis == 2
            x, y = i0 % nx, (i0 // nx) % ny
            uses[y, x] += 1
    assert np.allclose(grad[3], uses * (t - 1.0))
    assert np.allclose(grad[4], uses * (-t))
    assert np.count_nonzero(grad[:3]) == 0 and np.count_nonzero(grad[5:]) == 0


def test_dist_loss_closed_form_and_gradient():
    # original surface z = c of a linear field: trilinear interpolation is
    # exact, |grad F| = 1, so the distance is |p_z - c|
    nx, ny, nz = 8, 8, 8
    c = 3.4
    f = synth.plane_field((nx, ny, nz), (0, 0, 1), c)
    g = np.random.Generator(np.random.PCG64(3))
    pts = g.uniform(0.5, 6.5, size=(50, 3))
    L, grad = oracle.dist_loss(f, 0.0, pts)
    fz = (pts[:, 2] - c).astype(np.float64)
    assert abs(L - np.mean(np.abs(fz))) < 1e-5
    assert np.allclose(grad[:, 2], np.sign(fz) / len(pts), atol=1e-9)
    assert np.allclose(grad[:, :2], 0.0, atol=1e-9)


def test_dist_loss_gradient_matches_finite_differences():
    f = synth.turbulence(16, seed=9)
    g = np.random.Generator(np.random.PCG64(4))
    pts = g.uniform(1.2, 13.8, size=(40, 3))
    pts += 0.03  # keep away from cell faces, where the trilinear gradient jumps
    L, grad = oracle.dist_loss(f, 0.1, pts)
    h = 1e-6
    for v in range(0, 40, 3):
        for a in range(3):
            pp, pm = pts.copy(), pts.copy()
            pp[v, a] += h
            pm[v, a] -= h
            if np.floor(pp[v, a]) != np.floor(pm[v, a]):
                continue
            fd = (oracle.dist_loss(f, 0.1, pp, False)[0] - oracle.dist_loss(f, 0.1, pm, False)[0]) / (2 * h)
            assert abs(fd - grad[v, a]) <= 1e-6 + 1e-5 * abs(fd), (v, a, fd, grad[v, a])


def test_composed_loss_gradient_matches_finite_differences():
    # L(f) = mean distance of the mesh of f to the surface of an original
    # field; dL/df = mc_backward(f, k, dist_loss'(positions))
    f0 = synth.turbulence(18, seed=11)
    f = (f0 + 0.1 * synth.uniform_noise(f0.shape, 12)).astype(np.float32)
    k = 0.0
    m = oracle.mc(f, k)
    L, gp = oracle.dist_loss(f0, k, m.pos.reshape(-1, 3))
    grad = oracle.mc_backward(f, k, gp.reshape(m.pos.shape))
    h = 1e-4
    nz, ny, nx = f.shape
    P = m.pos.reshape(-1, 3)
    E = m.edge_id.reshape(-1)
    steps = (1, nx, nx * ny)
    checked = 0
    for (z, y, x) in _safe_vertices(f, k, h, 40, 6):
        # |F(p) - k| has a kink at the original surface: skip vertices that
        # move a mesh point within reach of it
        i = x + nx * (y + ny * z)
        near = [j for j in range(E.size) if E[j] // 3 == i or E[j] // 3 + steps[E[j] % 3] == i]
        if any(oracle.dist_loss(f0, k, P[j:j + 1], False)[0] < 0.02 for j in near):
            continue
        checked += 1
        fp, fm = f.copy(), f.copy()
        fp[z, y, x] += np.float32(h)
        fm[z, y, x] -= np.float32(h)
        Lp = oracle.dist_loss(f0, k, oracle.mc(fp, k).pos.reshape(-1, 3), False)[0]
        Lm = oracle.dist_loss(f0, k, oracle.mc(fm, k).pos.reshape(-1, 3), False)[0]
        fd = (Lp - Lm) / (float(fp[z, y, x]) - float(fm[z, y, x]))
        assert abs(fd - grad[z, y, x]) <= 1e-9 + 1e-3 * abs(fd), (z, y, x, fd, grad[z, y, x])
    assert checked >= 5
