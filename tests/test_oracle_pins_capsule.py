"""Pins of the oracle's proxy capsules and avatar queries (Sec. 3.3.2 dynamic
NavMesh blocking, Sec. 3.4 query APIs): capsule endpoints against the rest pose
and a rigid motion, distances and first contacts against brute-force sampling.
CPU only."""
import numpy as np

from paper_2604_12626_gb300 import synth


def _seg_dist_brute(p, a, b, n=200_001):
    t = np.linspace(0.0, 1.0, n)[:, None]
    return np.sqrt(((a[None] + t * (b - a)[None] - p[None]) ** 2).sum(1)).min()


def test_capsules_of_rest_pose_and_rigid_motion(oracle):
    rest, parents = synth.REST_JOINTS.astype(np.float64), synth.PARENTS
    J = rest.shape[0]
    radius = np.linspace(0.05, 0.12, J)
    # identity skinning matrices: each capsule spans the rest parent and joint
    M = np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]), (1, J, 1, 1))
    caps = oracle.avatar_capsules(M, rest, parents, radius)[0]
    for j in range(J):
        pj = parents[j] if parents[j] >= 0 else j
        np.testing.assert_allclose(caps[j, :3], rest[pj], atol=1e-15)
        np.testing.assert_allclose(caps[j, 4:7], rest[j], atol=1e-15)
        assert caps[j, 3] == radius[j]
    # one rigid transform for every joint moves every endpoint by it
    rng = np.random.default_rng(0)
    Rm = synth.rodrigues(rng.normal(0, 1, 3))
    tv = rng.normal(0, 1, 3)
    M2 = np.tile(np.hstack([Rm, tv[:, None]]), (1, J, 1, 1))
    caps2 = oracle.avatar_capsules(M2, rest, parents, radius)[0]
    np.testing.assert_allclose(caps2[:, :3], caps[:, :3] @ Rm.T + tv, atol=1e-12)
    np.testing.assert_allclose(caps2[:, 4:7], caps[:, 4:7] @ Rm.T + tv, atol=1e-12)


def test_distance_and_nearest_against_sampling(oracle):
    rng = np.random.default_rng(1)
    caps = np.zeros((2, 5, 8))
    caps[..., :3] = rng.uniform(0, 3, (2, 5, 3))
    caps[..., 4:7] = caps[..., :3] + rng.normal(0, 0.4, (2, 5, 3))
    caps[..., 3] = rng.uniform(0.05, 0.2, (2, 5))
    caps[0, 2, 4:7] = caps[0, 2, :3]  # a sphere (degenerate segment)
    off = np.array([0, 5, 10])
    Q = 40
    qe = rng.integers(0, 2, Q).astype(np.int32)
    p0 = rng.uniform(-0.5, 3.5, (Q, 3))
    out = oracle.capsule_query(caps.reshape(-1, 8), off, qe, p0)
    for q in range(Q):
        c = caps[qe[q]]
        d = np.array([_seg_dist_brute(p0[q], c[k, :3], c[k, 4:7]) - c[k, 3] for k in range(5)])
        L = np.linalg.norm(c[:, 4:7] - c[:, :3], axis=1).max()
        k = int(np.argmin(d))
        assert out["nearest"][q] == k
        # the exact distance is the infimum: at most the sampled one, and within the sampling step
        assert d[k] - L / 2e5 - 1e-12 <= out["dist"][q] <= d[k] + 1e-12
        assert out["tclip"][q] == (0.0 if out["blocked"][q] else 1.0)  # no step: contact only at the start
    # no capsules in an env: infinite distance, no nearest, never blocked
    none = oracle.capsule_query(caps.reshape(-1, 8)[:0], np.array([0, 0]), np.array([0], np.int32), p0[:1], p0[:1] + 1)
    assert none["nearest"][0] == -1 and np.isinf(none["dist"][0]) and not none["blocked"][0] and none["tclip"][0] == 1.0


def test_first_contact_against_sampling(oracle):
    rng = np.random.default_rng(2)
    n_caps, Q, r = 12, 60, 0.15
    caps = np.zeros((n_caps, 8))
    caps[:, :3] = rng.uniform(0, 2, (n_caps, 3))
    caps[:, 4:7] = caps[:, :3] + rng.normal(0, 0.5, (n_caps, 3))
    caps[:, 3] = rng.uniform(0.05, 0.15, n_caps)
    p0 = rng.uniform(-0.5, 2.5, (Q, 3))
    p1 = p0 + rng.normal(0, 1.0, (Q, 3))
    out = oracle.capsule_query(caps, np.array([0, n_caps]), np.zeros(Q, np.int32), p0, p1, agent_radius=r)
    t = np.linspace(0.0, 1.0, 20_001)
    n_blocked = 0
    for q in range(Q):
        pts = p0[q][None] + t[:, None] * (p1[q] - p0[q])[None]
        # distance of every sampled position to every capsule axis, minus its inflated radius
        f = np.full(t.size, np.inf)
        for k in range(n_caps):
            a, b = caps[k, :3], caps[k, 4:7]
            ab = b - a
            s = np.clip(((pts - a) @ ab) / (ab @ ab), 0.0, 1.0)
            f = np.minimum(f, np.linalg.norm(pts - (a + s[:, None] * ab), axis=1) - (caps[k, 3] + r))
        hit = np.flatnonzero(f <= 0.0)
        if hit.size == 0:
            # free: the sampled minimum stays above contact, unless it grazes within the sampling step
            assert not out["blocked"][q] or f.min() < 1e-4 * np.linalg.norm(p1[q] - p0[q])
            if not out["blocked"][q]:
                assert out["tclip"][q] == 1.0
            continue
        n_blocked += 1
        assert out["blocked"][q]
        k = hit[0]
        lo = t[k - 1] if k > 0 else 0.0
        assert lo - 1e-9 <= out["tclip"][q] <= t[k] + 1e-9, (q, out["tclip"][q], lo, t[k])
    assert 5 <= n_blocked <= Q - 5  # both outcomes are exercised


def test_step_starting_in_contact_and_tie_to_lowest_index(oracle):
    caps = np.array([[0, 0, 0, 0.2, 1, 0, 0, 0], [0, 0, 0, 0.2, 1, 0, 0, 0], [5, 5, 5, 0.1, 5, 5, 5, 0]], float)
    p0 = np.array([[0.5, 0.25, 0.0], [0.5, 1.0, 0.0]])
    p1 = np.array([[3.0, 3.0, 0.0], [0.5, -1.0, 0.0]])
    out = oracle.capsule_query(caps, np.array([0, 3]), np.zeros(2, np.int32), p0, p1, agent_radius=0.1)
    assert out["nearest"][0] == 0 and out["nearest"][1] == 0  # equal capsules 0 and 1: the lower index
    assert abs(out["dist"][0] - 0.05) < 1e-15 and out["blocked"][0] and out["tclip"][0] == 0.0
    # straight down onto the bone from y = 1: first contact at y = 0.2 + 0.1, t = 0.7 / 2
    assert out["blocked"][1] and abs(out["tclip"][1] - 0.35) < 1e-12
