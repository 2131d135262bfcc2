"""Counter-based random streams of the method, float64/integer NumPy oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper draws two kinds of random objects per mode (Sec. 3.1 and Alg. 1:
the fiber sample and the Gaussian sketch matrix):

* the sampling matrix E_k: s_k distinct canonical vectors of R^{n_{!=k}},
  picked uniformly at random with no repetition (Sec. 3.1 and its footnote);
* the Gaussian test matrix Omega_k in R^{s_k x (r_k+p)} (Sec. 3.1).

The paper fixes neither a generator nor a without-repetition sampler.  This
oracle (and, independently, the CUDA library) realises them from one published
counter-based generator so both sides draw the same numbers from a seed:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies, Weyl key schedule.
* A 4-round balanced Feistel network on [0, 2^b) whose round function is one
  Philox draw; restricted to [0, N) by cycle-walking (Black & Rogaway, "Ciphers
  with arbitrary finite domains", CT-RSA 2002).  Its first s outputs are s
  distinct indices of [0, N): the sample E_k.
* Box-Muller (Box & Muller 1958) turning two uniforms into one N(0,1) draw.
  Omega_k's entry (j, c) is keyed by the *linear fiber index* pi_k(j), not by
  the sample position j, so E_k Omega_k is the restriction of one dense
  Gaussian n_{!=k} x (r_k+p) matrix to the sampled rows (the dense Gaussian
  test matrix of R-HOSVD, Sec. 3, when s_k = n_{!=k}).

Stream separation: word 3 of the Philox counter is (stream << 16) | node with
stream 1 for the Feistel rounds, 2 for the Gaussians of the sketch and 3 for the
per-mode Gaussians of the Kronecker-structured sketch; ``node`` is the mode k
(Tucker) or the node id of the dimension tree (H-Tucker).  The key is the
64-bit seed split into two 32-bit words.
"""

import numpy as np

# Philox constants published in Salmon et al. (SC'11), Sec. 5 / Random123.
PHILOX4x32 = dict(W=32, M0=0xD2511F53, M1=0xCD9E8D57, W0=0x9E3779B9, W1=0xBB67AE85)
PHILOX4x64 = dict(W=64, M0=0xD2E7470EE14C6C93, M1=0xCA5A826395121157,
                  W0=0x9E3779B97F4A7C15, W1=0xBB67AE8584CAA73B)

STREAM_FEISTEL = 1
STREAM_GAUSS = 2
STREAM_KRON = 3     # the per-mode Gaussians of the Kronecker-structured sketch (oracle/rhkron.py)
TWO_PI = 6.283185307179586  # 2*pi rounded to float64
FEISTEL_ROUNDS = 4


def philox4(ctr, key, params=PHILOX4x32, rounds=10, scalar=False):
    """Philox4xW-R bijection (Salmon et al., SC'11, Sec. 5).

    ``ctr`` is a 4-tuple and ``key`` a 2-tuple of words.  For W=32 the words are
    NumPy uint64 arrays holding 32-bit values (vectorised) unless ``scalar``;
    for W=64 (or ``scalar``) they are Python ints.  One round maps (c0,c1,c2,c3) to
    (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)); the key is bumped
    by the Weyl constants (W0, W1) before every round but the first.
    """
    W = params["W"]
    mask = (1 << W) - 1
    M0, M1, W0, W1 = params["M0"], params["M1"], params["W0"], params["W1"]
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    if W == 32 and not scalar:
        m0, m1 = np.uint64(M0), np.uint64(M1)
        w0, w1 = np.uint64(W0), np.uint64(W1)
        msk = np.uint64(mask)
        sh = np.uint64(32)
        c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3))
        k0, k1 = np.uint64(k0), np.uint64(k1)

        def mulhilo(m, c):
            prod = m * c  # < 2^64: exact in uint64
            return prod >> sh, prod & msk
    else:
        m0, m1, w0, w1, msk = M0, M1, W0, W1, mask

        def mulhilo(m, c):
            prod = m * c
            return prod >> W, prod & msk
    for rnd in range(rounds):
        if rnd:
            k0 = (k0 + w0) & msk
            k1 = (k1 + w1) & msk
        hi0, lo0 = mulhilo(m0, c0)
        hi1, lo1 = mulhilo(m1, c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the two 32-bit Philox key words."""
    seed = int(seed) & ((1 << 64) - 1)
    return seed & 0xFFFFFFFF, seed >> 32


def feistel_bits(N):
    """Width b of the Feistel domain [0, 2^b): the smallest even b >= 2 with 2^b >= N."""
    N = int(N)
    b = max(2, (N - 1).bit_length())
    return b + (b & 1)


def feistel_permute(x, N, seed, node):
    """One pass of the keyed balanced Feistel bijection of [0, 2^b), b = feistel_bits(N).

    x = (L, R) with L the high and R the low h = b/2 bits; round t in 0..3 maps
    (L, R) -> (R, L xor (F_t(R) mod 2^h)), F_t(R) = word 0 of
    Philox4x32-10(ctr = (R, t, 0, (1 << 16) | node), key = seed).
    """
    b = feistel_bits(N)
    h = b // 2
    hmask = np.uint64((1 << h) - 1)
    k0, k1 = seed_key(seed)
    x = np.asarray(x, dtype=np.uint64)
    L = x >> np.uint64(h)
    R = x & hmask
    zero = np.zeros_like(R)
    w3 = np.uint64((STREAM_FEISTEL << 16) | int(node))
    for t in range(FEISTEL_ROUNDS):
        f = philox4((R, zero + np.uint64(t), zero, zero + w3), (k0, k1))[0]
        L, R = R, L ^ (f & hmask)
    return (L << np.uint64(h)) | R


def fiber_indices(N, s, seed, node):
    """pi(j), j = 0..s-1: s distinct indices of [0, N), uniform without repetition.

    Realises the sampling matrix E of Sec. 3.1 (s_k canonical basis vectors of
    R^{n_{!=k}} drawn uniformly, none twice).  Cycle-walking: y = P(j); while
    y >= N: y = P(y).  Since P permutes [0, 2^b), the walk restricted to [0, N)
    is a permutation of [0, N), so distinct j give distinct pi(j).
    """
    N, s = int(N), int(s)
    if not (0 <= s <= N):
        raise ValueError("need 0 <= s <= N")
    y = feistel_permute(np.arange(s, dtype=np.uint64), N, seed, node)
    out = y.copy()
    todo = out >= np.uint64(N)
    while np.any(todo):
        out[todo] = feistel_permute(out[todo], N, seed, node)
        todo = out >= np.uint64(N)
    return out.astype(np.int64)


def gaussian(m, c, seed, node, stream=None):
    """N(0,1) entries g(seed, node, m, c) by Box-Muller, float64.

    (u0, u1) = first two words of Philox4x32-10(ctr = (m mod 2^32, m >> 32, c,
    (2 << 16) | node), key = seed); a = (u0 + 1/2) 2^-32, b = (u1 + 1/2) 2^-32
    (both in (0, 1)); g = sqrt(-2 ln a) cos(2 pi b).  ``m`` and ``c`` broadcast.
    ``stream`` replaces the 2 in word 3 (default: the sketch's stream).
    """
    if stream is None:
        stream = STREAM_GAUSS
    m = np.asarray(m, dtype=np.uint64)
    c = np.asarray(c, dtype=np.uint64)
    m, c = np.broadcast_arrays(m, c)
    k0, k1 = seed_key(seed)
    lo = m & np.uint64(0xFFFFFFFF)
    hi = m >> np.uint64(32)
    w3 = np.zeros_like(m) + np.uint64((int(stream) << 16) | int(node))
    u0, u1, _, _ = philox4((lo, hi, c, w3), (k0, k1))
    a = (u0.astype(np.float64) + 0.5) * 2.0 ** -32
    b = (u1.astype(np.float64) + 0.5) * 2.0 ** -32
    return np.sqrt(-2.0 * np.log(a)) * np.cos(TWO_PI * b)


def sketch_matrix(pi, ncols, seed, node):
    """Omega (len(pi) x ncols): Omega[j, c] = g(seed, node, pi[j], c) (Sec. 3.1, Alg. 1)."""
    pi = np.asarray(pi, dtype=np.uint64)
    cols = np.arange(ncols, dtype=np.uint64)
    return gaussian(pi[:, None], cols[None, :], seed, node)
