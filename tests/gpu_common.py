"""Shared helpers of the GPU parity tests: oracle results for a suspension of a workload."""
import numpy as np

from oracle import forces, geometry as G, rigid, rpy
from oracle.gdc import Params as OParams


def susp_layout(wl, s):
    off = wl.susp_body_off
    bt = wl.body_tmpl[off[s]:off[s + 1]]
    return G.Layout(wl.templates, bt), wl.Y[off[s]:off[s + 1]], wl.q[off[s]:off[s + 1]]


def blob_slices(wl):
    nb = wl.tmpl_nblobs[wl.body_tmpl]
    boff = np.concatenate([[0], np.cumsum(nb)])
    return [(int(boff[wl.susp_body_off[s]]), int(boff[wl.susp_body_off[s + 1]])) for s in range(wl.n_susp)]


def oracle_params(wl, **kw):
    pp = dict(wl.params)
    pp.update(kw)
    return OParams.from_dict(pp)


def dense_state(lay, Y, q, a=1.0, eta=1.0):
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, a, eta)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    B = rigid.rigid_basis(K, lay.n_bodies)
    return r, M, K, B


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rot_err(q1, q2):
    return max(float(np.linalg.norm(G.rotation_matrix(a) - G.rotation_matrix(b))) for a, b in zip(q1, q2))


def saddle_vec(wl, lam_list, V_list):
    """Stack per-suspension [lambda; V] blocks into the library's saddle layout."""
    return np.concatenate([np.concatenate([l.reshape(-1), v.reshape(-1)]) for l, v in zip(lam_list, V_list)])


def split_saddle(wl, x):
    out = []
    pos = 0
    for s in range(wl.n_susp):
        lay, _, _ = susp_layout(wl, s)
        nl, nv = 3 * lay.n_blobs, 6 * lay.n_bodies
        out.append((x[pos:pos + nl], x[pos + nl:pos + nl + nv]))
        pos += nl + nv
    return out
