"""The near-contact film measurement from sign masks (the GPU pass's NcRay::measure)
against the sequential march over the same samples (NcMarch::feed, the oracle's
order), on the host: both restated here from the kernel's rules, on random sample
sequences with unsigned samples (|v| <= 1e-5), crossings at every position and films
of every length. The GPU pass computes the samples themselves exactly as the march
does; this checks that the mask rules decide A_h as the march does on any sequence.
"""
import numpy as np

BAND = 1e-5


def A_h(h, A=0.02, h_min=3.0, h_cut=6.0):
    if h <= h_min:
        return A
    if h >= h_cut:
        return 0.0
    b3 = (h_min / h_cut) ** 3
    return A * ((h_min / h) ** 3 - b3) / (1.0 - b3)


def t_of(s):
    return -1.0 + 0.5 * s


def march(v, h_cut=6.0):
    """Samples in order: the first downward crossing, the first upward one after it;
    stop with 0 at a signed sample at least h_cut past the downward crossing."""
    have_a = have_d = False
    t_a = v_a = t_d = 0.0
    for s, vs in enumerate(v):
        t = t_of(s)
        if abs(vs) <= BAND:
            continue
        if have_a:
            if not have_d and v_a > 0 and vs < 0:
                t_d = t_a + (t - t_a) * v_a / (v_a - vs)
                have_d = True
            elif have_d and v_a < 0 and vs > 0:
                t_u = t_a + (t - t_a) * v_a / (v_a - vs)
                return A_h(t_u - t_d, h_cut=h_cut)
        if have_d and t - t_d >= h_cut:
            return 0.0
        t_a, v_a, have_a = t, vs, True
    return 0.0


def masks(v, h_cut=6.0):
    """The kernel's rules: j = the first negative sample whose previous signed sample
    is positive (jp), k = the first positive sample after j, kp its previous signed
    sample; 0 when kp != j and t_kp - t_d >= h_cut."""
    P = sum(1 << s for s, x in enumerate(v) if x > BAND)
    N = sum(1 << s for s, x in enumerate(v) if x < -BAND)
    S = P | N
    jp = j = -1
    prev = None
    m = S
    while m:
        i = (m & -m).bit_length() - 1
        m &= m - 1
        if prev is not None and (P >> prev) & 1 and (N >> i) & 1:
            jp, j = prev, i
            break
        prev = i
    if j < 0:
        return 0.0
    later = P & ~((2 << j) - 1)
    if not later:
        return 0.0
    k = (later & -later).bit_length() - 1
    kp = (S & ((1 << k) - 1)).bit_length() - 1
    t_d = t_of(jp) + (t_of(j) - t_of(jp)) * v[jp] / (v[jp] - v[j])
    if kp != j and t_of(kp) - t_d >= h_cut:
        return 0.0
    t_u = t_of(kp) + (t_of(k) - t_of(kp)) * v[kp] / (v[kp] - v[k])
    return A_h(t_u - t_d, h_cut=h_cut)


def test_masks_decide_as_the_march():
    rng = np.random.default_rng(11)
    films = 0
    for n in range(20000):
        kind = n % 4
        if kind == 0:      # smooth profiles: a droplet edge, a film, another droplet
            a, b = sorted(rng.uniform(-1.0, 9.0, size=2))
            t = np.array([t_of(s) for s in range(19)])
            v = np.tanh(2.0 * (a - t)) + np.tanh(2.0 * (t - b)) + rng.uniform(-0.9, 0.9)
        elif kind == 1:    # random signs with unsigned samples sprinkled in
            v = rng.choice([-1.0, 1.0], size=19) * rng.uniform(0.0, 1.0, size=19)
            v[rng.random(19) < 0.2] = rng.uniform(-BAND, BAND)
        elif kind == 2:    # values at the band's edges
            v = rng.choice([-1.0, 1.0], size=19) * rng.choice([0.5 * BAND, BAND, 2 * BAND, 0.3], size=19)
        else:              # mostly negative with short positive runs
            v = -rng.uniform(0.01, 1.0, size=19)
            for _ in range(rng.integers(0, 4)):
                s0 = rng.integers(0, 19)
                v[s0:s0 + rng.integers(1, 4)] = rng.uniform(0.01, 1.0)
        v = [float(x) for x in v]
        want, got = march(v), masks(v)
        assert got == want, (v, want, got)
        films += want > 0
    assert films > 1000
