"""Element-wise tolerances of the closure network's tensor-core path against
the FP64 oracle of oracle/closure.py (test helper, no GPU needed).

The kernels store inputs, weights, hidden activations and the back-propagated
signal in bf16 and accumulate in fp32.  The oracle with emulate_bf16=True
rounds to bf16 at exactly those points and accumulates in FP64, so the two
differ only by
  * the fp32 accumulation order: a K = 576-term dot product carries a
    relative error of at most K 2^-24 = 3.4e-5 of the sum of its absolute
    terms (about sqrt(K) 2^-24 = 1.4e-6 in practice);
  * the bf16 values that this tiny difference moves across a rounding
    boundary: such a value lands on the neighbouring bf16 number, a change
    of 2^-8 of itself, which then feeds the layers after it.
A network output is a 576-term sum of products of the last hidden layer, so
one such neighbouring-value flip moves it by at most 2^-8 of its largest
term, far less relative to the output; FWD_RTOL = 2 * 2^-8 allows two flips
at full size.  A gradient element is a sum over every pixel of the batch
(768 to 1024 terms) that cancels strongly, and flips in the activations and
in the ReLU masks move it by a few per mille of the layer's rms each:
GRAD_RTOL = 4e-2 of max(|g|, rms of the layer's tensor), about twice the
largest element seen on random and on realistic data; per layer the
relative L2 difference stays below GRAD_LAYER_L2 = 1e-2 (seen: <= 3e-3).

Where the residual y - t is small and its column means are taken out (the
output centring, which removes the column-mean part of dL/dy), the gradient
elements cancel far more and those flips weigh more: on the oracle's own
moving-average targets, jittering every pre-activation by 2e-6 of its rms
(the size of an fp32 reordering) moves single weight-gradient elements of
the oracle itself by up to ~0.2 of the layer's rms.  decision_spread()
measures that spread on the test's own data, with the oracle alone; a layer
may then differ by up to twice the largest spread seen, where that is above
GRAD_RTOL (and the per-layer relative L2 likewise).

Against the exact FP64 network (no bf16 rounding) the GPU can be no closer
than the bf16 definition itself, which the oracle measures on its own
(emulating versus exact: forward ~0.3-0.6 %, first-layer weight gradient
5-8 % relative L2, from the rounding of the signal back-propagated through
three layers); the tests check that the GPU is no further from the exact
network than that plus the accumulation-order term.
"""
import numpy as np

FWD_RTOL = 2.0 * 2.0 ** -8
GRAD_RTOL = 4e-2
GRAD_LAYER_L2 = 1e-2


def rms(b) -> float:
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.mean(b * b))) if b.size else 0.0


def elem_err(a, b, scale=None) -> float:
    """max |a - b| / max(|b|, scale), scale = rms(b) unless given."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = rms(b) if scale is None else scale
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), max(s, 1e-300))))


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_patches(steps: int = 400, seed: int = 3):
    """Realistic network inputs and targets from the oracle's own coupled run
    (feedback = 2: sampling only, no imposition): a 64 x 18 D2Q9 channel with
    MPCD on the 16 central columns at r = 2 (32 x 32 fine cells, ppc 10,
    kT 1e-4, g 2e-6); CLOSURE_IN and CLOSURE_TARGET after `steps` steps, four
    16 x 16 patches.  Binary32-rounded, as the GPU receives them."""
    import oracle
    p = dict(lattice=9, nx=64, ny=18, nz=1, tau=0.8, force=(2e-6, 0.0, 0.0), refine=2, ppc=10,
             alpha=np.radians(130.0), kT=1e-4, mass=1.0, coupling_width=2, precision=0, feedback=2,
             window=100, resample_density=0, seed=seed)
    s = oracle.OracleSim(p)
    s.set_region(16, 48)
    s.step(steps)
    x = s.get("CLOSURE_IN").reshape(-1, 16, 16, 24).astype(np.float32).astype(np.float64)
    t = s.get("CLOSURE_TARGET").reshape(-1, 16, 16, 3).astype(np.float32).astype(np.float64)
    return x, t


def decision_spread(C, th, x, t, draws: int = 4, rel: float = 2e-6, seed: int = 0):
    """Per-layer [(W elem, W L2, b elem, b L2)]: the largest element error
    (elem_err against the layer's rms) and relative L2 by which the oracle's
    bf16-emulating gradient moves when every pre-activation is jittered by
    `rel` of its rms (normal draws): the sensitivity of the bf16 and ReLU
    decisions to the accumulation order, measured on the oracle alone."""
    rng = np.random.default_rng(seed)
    _, g0 = C.backward(th, x, t, emulate_bf16=True)
    out = np.zeros((len(C.LAYERS), 4))
    for _ in range(draws):
        _, g = C.backward(th, x, t, emulate_bf16=True,
                          jitter=lambda z: z + rel * rms(z) * rng.normal(size=z.shape))
        o = 0
        for li, (ci, co) in enumerate(C.LAYERS):
            nW = co * 9 * ci
            for k, sl in enumerate((slice(o, o + nW), slice(o + nW, o + nW + co))):
                out[li, 2 * k] = max(out[li, 2 * k], elem_err(g[sl], g0[sl], rms(g0[sl])))
                out[li, 2 * k + 1] = max(out[li, 2 * k + 1], rel_l2(g[sl], g0[sl]))
            o += nW + co
    return out
