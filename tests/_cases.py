"""Small shared test inputs (geometry only)."""
import numpy as np

from paper_2603_28475_b300 import scenes as S
from oracle import geometry as G

MM = 1e-3


def f32(v):
    """The value a float parameter has once it crosses the C ABI (float32)."""
    return float(np.float32(v))


def oracle_pad(pd, mat):
    """Oracle model of a scene pad with the material values the library
    receives (float32 fields of tac_params)."""
    return G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, f32(mat.E), f32(mat.nu), f32(mat.rho), f32(mat.h),
                       f32(mat.dhat), f32(mat.mu_f))


def tiny_pad(cells=(2, 2, 1), size=(4 * MM, 4 * MM, 2 * MM), E=0.3e6, nu=0.45, mu_f=0.0, jitter=0.0, seed=0):
    pd = S.hex_pad(size, cells, marker_shape=(3, 3), jitter=jitter, rng=np.random.default_rng(seed))
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, E, nu, 1100.0, 1 / 60, 0.05 * MM, mu_f)
    return pd, pad


def small_indenter(radius=1.5 * MM, subdiv=1):
    ind = S.icosphere(radius, subdiv)
    return ind, G.build_indenter(ind.verts, ind.tris)


def c1():
    w = S.config_single_pad()
    pad = oracle_pad(w.pads[0], w.materials[0])
    ind = G.build_indenter(w.indenters[0].verts, w.indenters[0].tris)
    return w, pad, ind
