"""GPU-vs-oracle comparison with the acceptance tolerances of the evaluation:

  positions (link p, sphere centres), rotations, d_min   |delta| <= 1e-5
  worst pair      equal, or the GPU's pair has an FP64 distance within 2e-5 m
                  of the oracle's d_min (near-ties)
  torques         ||delta tau||_inf <= 1e-4 * max(||tau_ref||_inf, 1 N m)
                  per configuration
  pair bits       equal for every pair with |d_ref| > 1e-5 m
  gradients       ||g - g_ref||_2 <= 1e-3 * max(||g_ref||_2, 1e-6) per
                  configuration for each of q_bar, qd_bar, qdd_bar, over the
                  configurations whose worst pair agrees with the oracle's
"""
import numpy as np

POS_TOL = 1e-5
TIE_TOL = 2e-5
TAU_REL = 1e-4
GRAD_REL = 1e-3


def pair_distances(desc, sph):
    """FP64 distances of every masked pair from sphere centres [B][S][3]."""
    i, j = desc.pairs[:, 0], desc.pairs[:, 1]
    diff = sph[:, i, :] - sph[:, j, :]
    return np.sqrt((diff ** 2).sum(-1)) - desc.sph_r[i] - desc.sph_r[j]


def check_forward(desc, got, ref, bits_ref_d=None, sample=None):
    """got: numpy outputs of the GPU (keys pose, sphere, dmin, worst, tau, bits);
    ref: oracle.evaluate output.  `sample` selects config indices of `got`
    that `ref` covers (ref is indexed 0..len(sample)-1)."""
    sel = slice(None) if sample is None else sample
    if got.get("pose") is not None:
        d = np.abs(got["pose"][sel] - ref["pose"]).max()
        assert d <= POS_TOL, "pose error %g" % d
    if got.get("sphere") is not None:
        d = np.abs(got["sphere"][sel] - ref["sph"]).max()
        assert d <= POS_TOL, "sphere error %g" % d
    if got.get("dmin") is not None and desc.P > 0:
        gd = got["dmin"][sel]
        d = np.abs(gd - ref["dmin"]).max()
        assert d <= POS_TOL, "d_min error %g" % d
        gw = got["worst"][sel]
        same = gw == ref["worst"]
        if not same.all():
            # near-ties: the GPU's pair must be within TIE_TOL of the minimum
            D = pair_distances(desc, ref["sph"])
            bad = [b for b in np.nonzero(~same)[0]
                   if not (0 <= gw[b] < desc.P and D[b, gw[b]] - ref["dmin"][b] <= TIE_TOL)]
            assert not bad, "worst pair differs at %s" % bad[:5]
    elif got.get("dmin") is not None:
        assert np.isinf(got["dmin"][sel]).all() and (got["worst"][sel] == -1).all()
    if got.get("tau") is not None:
        t = got["tau"][:, sel]
        err = np.abs(t - ref["tau"]).max(axis=0)
        scale = np.maximum(np.abs(ref["tau"]).max(axis=0), 1.0)
        worst = (err / scale).max()
        assert worst <= TAU_REL, "tau rel error %g" % worst
    if got.get("bits") is not None and desc.P > 0:
        W = (desc.P + 31) // 32
        words = got["bits"][sel][:, :W].astype(np.uint32)
        bits = np.unpackbits(words.view(np.uint8).reshape(words.shape[0], -1),
                             axis=1, bitorder="little")[:, :desc.P].astype(bool)
        D = pair_distances(desc, ref["sph"])
        firm = np.abs(D) > POS_TOL
        assert np.array_equal(bits[firm], (D < 0)[firm]), "pair bits differ"


def check_gradient(got, ref, mask=None):
    """got, ref: (gq, gqd, gqdd) each [d][B]; mask: configs to compare."""
    for name, g, r in zip(("q", "qd", "qdd"), got, ref):
        if mask is not None:
            g, r = g[:, mask], r[:, mask]
        err = np.linalg.norm(g - r, axis=0)
        nrm = np.maximum(np.linalg.norm(r, axis=0), 1e-6)
        worst = (err / nrm).max() if err.size else 0.0
        assert worst <= GRAD_REL, "grad %s rel error %g" % (name, worst)


def stable_seed(*parts) -> int:
    """A seed in [0, 1000) from test parameters, the same in every process
    (Python's str hash is salted per process)."""
    import zlib
    return zlib.crc32(repr(parts).encode()) % 1000
