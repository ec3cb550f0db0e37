"""Pins of the oracle against what the standard and the mathematics fix.

Each test names the passage it checks.  None of them re-types the oracle's
formula: they check a consequence (a derived index map, a diffusion pattern, a
bijection, an algebraic identity) that a plausible mistake would break.
"""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _unit(w, x, y, z):
    S = np.zeros(25 * w, dtype=np.uint8)
    S[w * (5 * y + x) + z] = 1  # Eq. 1
    return S


def _ones(S, w):
    idx = np.flatnonzero(S)
    return sorted((int(i // w) % 5, int(i // w) // 5, int(i % w)) for i in idx)


# -- Table 1 ------------------------------------------------------------------
def test_width_table_matches_table1(oracle_mod):
    rows = [tuple(map(int, ln.split())) for ln in open(os.path.join(HERE, "golden", "table1_widths.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 7
    for b, w, l in rows:
        assert b == 25 * w and 2 ** l == w
        # Keccak-p[b, 12+2l] accepts exactly the Table 1 widths.
        oracle_mod.keccak_p(b, 12 + 2 * l, np.zeros(b, dtype=np.uint8))
        # Its RC lane has bits only at 2^j - 1, j = 0..l (Eq. 8).
        for ir in range(12 + 2 * l):
            rc = oracle_mod.round_constant(l, ir)
            assert rc & ~sum(1 << (2 ** j - 1) for j in range(l + 1)) == 0
    for bad in (75, 3200):
        with pytest.raises(ValueError):
            oracle_mod.keccak_p(bad, 1, np.zeros(bad, dtype=np.uint8))


# -- rc and iota (Definition 5, Eq. 8-9) --------------------------------------
def test_rc_is_the_lfsr_polynomial(oracle_mod):
    # rc(t) is the constant term of x^t mod (x^8 + x^6 + x^5 + x^4 + 1) over
    # GF(2): the polynomial statement of FIPS 202 Algorithm 5's register.
    poly = (1 << 8) | (1 << 6) | (1 << 5) | (1 << 4) | 1
    v = 1
    for t in range(0, 600):
        assert oracle_mod.rc_bit(t) == (v & 1), t
        v <<= 1
        if v & 0x100:
            v ^= poly
    for t in range(-300, 0):  # t mod 255, taken non-negative
        assert oracle_mod.rc_bit(t) == oracle_mod.rc_bit(t % 255)


def test_round_constants_from_rc(oracle_mod):
    # 24 rounds of Keccak-f[1600]: bit 2^j - 1 of RC is rc(j + 7 i_r), j = 0..6.
    for ir in range(24):
        rc = oracle_mod.round_constant(6, ir)
        for j in range(7):
            assert (rc >> (2 ** j - 1)) & 1 == oracle_mod.rc_bit(j + 7 * ir)


def test_iota_touches_lane_00_only(oracle_mod):
    rng = np.random.default_rng(5)
    for w, l in ((1, 0), (8, 3), (64, 6)):
        S = rng.integers(0, 2, size=25 * w, dtype=np.uint8)
        for ir in (0, 3, 11):
            out = oracle_mod.step("iota", w, S, ir)
            diff = out ^ S
            assert not diff[w:].any()
            rc = oracle_mod.round_constant(l, ir)
            assert [int(b) for b in diff[:w]] == [(rc >> z) & 1 for z in range(w)]


# -- rho (Definition 2, Eq. 5) and pi (Definition 3, Eq. 6) -------------------
def test_rho_walk_and_offsets(oracle_mod):
    # The walk (x, y) -> (y, 2x + 3y mod 5) from (1, 0) is one cycle through the
    # 24 lanes other than (0, 0), and the 25 offsets are distinct mod 64.
    seen, (x, y) = [], (1, 0)
    for _ in range(24):
        seen.append((x, y))
        x, y = y, (2 * x + 3 * y) % 5
    assert (x, y) == (1, 0) and len(set(seen)) == 24 and (0, 0) not in seen
    offs = [oracle_mod.rho_offset(64, x, y) for y in range(5) for x in range(5)]
    assert offs[0] == 0 and len(set(offs)) == 25


@pytest.mark.parametrize("w", (1, 2, 8, 64))
def test_rho_rotates_within_lane(oracle_mod, w):
    # A single bit stays in its lane and moves from z to z + offset (mod w):
    # rotation towards higher z, i.e. a left rotate of the lane word.
    for x in range(5):
        for y in range(5):
            off = oracle_mod.rho_offset(w, x, y)
            for z in {0, w - 1, w // 2}:
                out = oracle_mod.step("rho", w, _unit(w, x, y, z))
                assert _ones(out, w) == [(x, y, (z + off) % w)]


@pytest.mark.parametrize("w", (1, 4, 64))
def test_pi_moves_lane_xy_to_y_2x3y(oracle_mod, w):
    # Eq. 6 pulls A'[x,y] from A[(x+3y) mod 5, x]; pushed forward, lane (x, y)
    # lands on (y, 2x + 3y mod 5) (3^-1 = 2 mod 5), with z unchanged.
    for x in range(5):
        for y in range(5):
            z = (3 * x + y) % w
            out = oracle_mod.step("pi", w, _unit(w, x, y, z))
            assert _ones(out, w) == [(y, (2 * x + 3 * y) % 5, z)]


# -- theta (Definition 1, Eq. 2-4) ---------------------------------------------
@pytest.mark.parametrize("w", (1, 2, 16, 64))
def test_theta_single_bit_diffusion(oracle_mod, w):
    # One bit at (x0, y0, z0) feeds C[x0, z0], hence D[x0+1, z0] and
    # D[x0-1, z0+1]: the output is the bit itself plus two whole columns,
    # 11 bits in all.
    for x0, y0, z0 in ((0, 0, 0), (2, 3, w - 1), (4, 1, w // 2), (1, 4, 1 % w)):
        out = oracle_mod.step("theta", w, _unit(w, x0, y0, z0))
        want = {(x0, y0, z0)}
        want |= {((x0 + 1) % 5, y, z0) for y in range(5)}
        want |= {((x0 - 1) % 5, y, (z0 + 1) % w) for y in range(5)}
        assert _ones(out, w) == sorted(want)


# -- chi (Definition 4, Eq. 7) ---------------------------------------------------
def test_chi_row_behaviour(oracle_mod):
    w = 4
    # A lone 1 at row position k: bit k stays and bit k-2 turns on, because
    # bit k-2 sees (not a[k-1]) and a[k].  Other rows and slices stay zero.
    for k in range(5):
        out = oracle_mod.step("chi", w, _unit(w, k, 2, 3))
        assert _ones(out, w) == sorted({(k, 2, 3), ((k - 2) % 5, 2, 3)})
    # chi acts on each 5-bit row as a bijection.
    images = set()
    for v in range(32):
        S = np.zeros(25 * w, dtype=np.uint8)
        for x in range(5):
            S[w * (5 * 1 + x) + 2] = (v >> x) & 1
        out = oracle_mod.step("chi", w, S)
        assert _ones(out, w) == [p for p in _ones(out, w) if p[1] == 1 and p[2] == 2]
        images.add(tuple(out[w * (5 * 1 + x) + 2] for x in range(5)))
    assert len(images) == 32


# -- the round and Keccak-p[b, n_r] (Eq. 10, FIPS 202 Algorithm 7) ------------
def test_keccak_p_round_indices(oracle_mod):
    rng = np.random.default_rng(7)
    for b, nr in ((1600, 24), (1600, 12), (200, 18), (200, 5), (25, 14)):
        w = b // 25
        l = int(np.log2(w))
        S = rng.integers(0, 2, size=b, dtype=np.uint8)
        ref = S.copy()
        for ir in range(12 + 2 * l - nr, 12 + 2 * l):  # the last n_r indices
            ref = oracle_mod.step("rnd", w, ref, ir)
        assert np.array_equal(oracle_mod.keccak_p(b, nr, S), ref), (b, nr)


def test_rnd_is_composition_in_eq10_order(oracle_mod):
    rng = np.random.default_rng(8)
    w = 8
    S = rng.integers(0, 2, size=25 * w, dtype=np.uint8)
    t = S
    for name in ("theta", "rho", "pi", "chi"):
        t = oracle_mod.step(name, w, t)
    t = oracle_mod.step("iota", w, t, 5)
    assert np.array_equal(oracle_mod.step("rnd", w, S, 5), t)


# -- bijectivity of the reduced permutations -----------------------------------
def test_keccak_f25_is_a_bijection_brute_force(oracle_mod):
    # All 2^25 states through Keccak-f[25] = Keccak-p[25, 12]: every image hit.
    assert oracle_mod.count_images_b25(12) == 2 ** 25


def _gf2_rank_and_inverse(M):
    n = M.shape[0]
    A = np.concatenate([M.copy() % 2, np.eye(n, dtype=np.uint8)], axis=1)
    rank = 0
    for col in range(n):
        piv = next((r for r in range(rank, n) if A[r, col]), None)
        if piv is None:
            continue
        A[[rank, piv]] = A[[piv, rank]]
        for r in range(n):
            if r != rank and A[r, col]:
                A[r] ^= A[rank]
        rank += 1
    return rank, (A[:, n:] if rank == n else None)


def test_keccak_f50_stepwise_bijective_and_invertible(oracle_mod):
    w, b = 2, 50
    units = [np.eye(b, dtype=np.uint8)[i] for i in range(b)]
    # theta is GF(2)-linear with a full-rank matrix.
    T = np.stack([oracle_mod.step("theta", w, u) for u in units], axis=1)
    rng = np.random.default_rng(9)
    for _ in range(20):
        a = rng.integers(0, 2, size=b, dtype=np.uint8)
        c = rng.integers(0, 2, size=b, dtype=np.uint8)
        assert np.array_equal(oracle_mod.step("theta", w, a ^ c),
                              oracle_mod.step("theta", w, a) ^ oracle_mod.step("theta", w, c))
    rank, T_inv = _gf2_rank_and_inverse(T)
    assert rank == b
    # rho and pi send unit vectors to distinct unit vectors: bit permutations.
    perms = {}
    for name in ("rho", "pi"):
        img = [int(np.flatnonzero(oracle_mod.step(name, w, u))[0]) for u in units]
        assert all(oracle_mod.step(name, w, u).sum() == 1 for u in units)
        assert sorted(img) == list(range(b))
        perms[name] = np.array(img)
    # chi: each row (x = 0..4 at fixed y, z) maps its 32 values injectively.
    chi_tab = np.zeros(32, dtype=np.int64)
    for v in range(32):
        S = np.zeros(b, dtype=np.uint8)
        for x in range(5):
            S[w * x] = (v >> x) & 1
        out = oracle_mod.step("chi", w, S)
        chi_tab[v] = sum(int(out[w * x]) << x for x in range(5))
    assert sorted(chi_tab) == list(range(32))
    chi_inv = np.argsort(chi_tab)
    # Round trip through an explicitly written inverse round.
    for trial in range(2000):
        ir = trial % 18
        A = rng.integers(0, 2, size=b, dtype=np.uint8)
        B = oracle_mod.step("rnd", w, A, ir)
        B = oracle_mod.step("iota", w, B, ir)  # iota is its own inverse
        rows = np.zeros(b, dtype=np.uint8)     # inverse chi, row by row
        for y in range(5):
            for z in range(w):
                v = sum(int(B[w * (5 * y + x) + z]) << x for x in range(5))
                u = chi_inv[v]
                for x in range(5):
                    rows[w * (5 * y + x) + z] = (u >> x) & 1
        before_pi = np.zeros(b, dtype=np.uint8)
        before_pi[np.arange(b)] = rows[perms["pi"]]
        before_rho = np.zeros(b, dtype=np.uint8)
        before_rho[np.arange(b)] = before_pi[perms["rho"]]
        back = (T_inv.astype(np.int64) @ before_rho.astype(np.int64)) % 2
        assert np.array_equal(back.astype(np.uint8), A), trial


# -- sponge (Section 3.2, FIPS 202 Algorithm 8) ---------------------------------
@pytest.mark.parametrize("variant,r", ((4, 168), (5, 136)))
def test_shake_prefix_consistency(oracle_mod, variant, r):
    msg = bytes(range(40))
    longest = oracle_mod.hash(variant, msg, 3 * r + 5)
    for d in (0, 1, r - 1, r, r + 1, 2 * r, 3 * r + 4):
        assert oracle_mod.hash(variant, msg, d) == longest[:d]


@pytest.mark.parametrize("variant", range(6))
def test_incremental_absorb_equals_one_shot(oracle_mod, variant):
    rng = np.random.default_rng(20 + variant)
    out_len = (28, 32, 48, 64, 100, 300)[variant]
    for L in (0, 1, 71, 72, 135, 136, 137, 350):
        msg = rng.integers(0, 256, size=L, dtype=np.uint8).tobytes()
        want = oracle_mod.hash(variant, msg, out_len)
        cuts = sorted(int(c) for c in rng.integers(0, L + 1, size=int(rng.integers(0, 5))))
        inc = oracle_mod.Incremental(variant)
        prev = 0
        for c in cuts + [L]:
            inc.absorb(msg[prev:c])
            prev = c
        assert inc.final(out_len) == want, (variant, L, cuts)


def test_keccak_c_on_bit_strings_equals_bytes_path(oracle_mod):
    # The byte API appends the suffix bits 0,1 after the LSB-first message bits
    # (FIPS 202 Appendix B); a message whose bit length is not a multiple of 8
    # goes through Keccak[c] directly and agrees with its byte-padded twin only
    # when the extra bits reproduce the suffix.
    msg = bytes([0xA5, 0x3C])
    bits = np.array([(byte >> j) & 1 for byte in msg for j in range(8)] + [0, 1], dtype=np.uint8)
    z = oracle_mod.keccak_c(512, bits, 256)
    packed = bytes(int(sum(int(z[8 * i + j]) << j for j in range(8))) for i in range(32))
    assert packed == oracle_mod.hash(1, msg)
