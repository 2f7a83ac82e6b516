"""Pins of the oracle's channel table and of its normalisation (CPU).

* The channel table: ids 0..51 must name the baryons of the paper's list
  (Sec. 4, Eqs. GeneralBB_NN .. GeneralBB_XX, printed order) and ids 52..55
  the four channels omitted there, transcribed in ``golden/channels.txt``.
  A swapped pair within a row or a misplaced row fails here, even where the
  diagram counts and quark contents of the neighbouring ids would agree.
* The normalisation R = C exp((m_B1 + m_B2) d) (Sec. 2 Eq. 2).  With one
  Gaussian draw G_f per flavour and propagators S_f = G_f exp(-m_f d), the
  raw correlator is C(d) = C(G) exp(-sum over the six sink quarks of m_f d),
  and flavour conservation makes the sink's quark content that of the
  source.  So R must not depend on d for any channel; it does only if the
  synthetic baryon mass of every sink baryon is the sum of its quark masses
  and the factor has the sign that undoes the decay.  This follows from the
  mathematics, not from the normalisation's own formula.
"""
import os

import numpy as np
import pytest

import synth
import oracle.oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))


def read_channels():
    rows = {}
    with open(os.path.join(HERE, "golden", "channels.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            cid, sink, src = (x.strip() for x in line.split("|"))
            rows[int(cid)] = tuple(sink.split()) + tuple(src.split())
    return rows


def test_channel_table_matches_the_printed_list():
    rows = read_channels()
    assert sorted(rows) == list(range(56))
    for cid, want in rows.items():
        assert orc.channel_baryons(cid) == want, (cid, orc.channel_baryons(cid), want)


def test_channel_table_rejects_a_swapped_source_pair():
    """The comparison is order-sensitive: B3 B4 swapped is a different entry."""
    rows = read_channels()
    b = orc.channel_baryons(2)  # p Lambda <- Sigma+ n
    assert b != rows[2][:2] + rows[2][2:][::-1]


def _slices(L, d, m_ud, m_s, seed):
    """S_f = G_f exp(-m_f d) with the same draws G_f for every d (u != d)."""
    V = L ** 3
    G = {s: synth.gaussian_slice(V, synth._slice_key(seed, 0, 0, k, 0))
         for s, k in (("u", synth.STREAM_LIGHT), ("d", synth.STREAM_DOWN), ("s", synth.STREAM_STRANGE))}
    return {"u": G["u"] * np.exp(-m_ud * d), "d": G["d"] * np.exp(-m_ud * d), "s": G["s"] * np.exp(-m_s * d)}


def _normalised_pair(L, chans, m_ud, m_s, d1, d2, seed=11):
    out = []
    for d in (d1, d2):
        S = _slices(L, d, m_ud, m_s, seed)
        C = orc.correlator(L, S["u"], S["d"], S["s"], chans)
        out.append(orc.normalise(C, chans, d, m_ud, m_s))
    return out


ALL_IDS = list(range(orc.n_channels()))


@pytest.mark.parametrize("ids", [ALL_IDS[:64], ALL_IDS[64:]], ids=["octet+charge", "decuplet"])
def test_normalised_correlator_does_not_depend_on_d(ids):
    L, m_ud, m_s = 1, 0.3, 0.4
    R1, R2 = _normalised_pair(L, ids, m_ud, m_s, 2, 7)
    for i, ch in enumerate(ids):
        scale = np.abs(R1[i]).max()
        assert scale > 0, ch
        assert np.abs(R1[i] - R2[i]).max() <= 1e-12 * scale, (ch, orc.channel_name(ch))


def test_normalisation_pin_catches_a_wrong_mass(monkeypatch):
    """Planted mistakes: one baryon's mass off, or the factor's sign flipped."""
    L, m_ud, m_s = 1, 0.3, 0.4
    ids = [1, 10, 42, 51]  # p Lambda, Lambda Lambda, Xi- Lambda, Xi- Xi0
    good = orc.baryon_mass

    def wrong_lambda(name, a, b):
        return good(name, a, b) + (0.05 if name == "Lambda" else 0.0)

    monkeypatch.setattr(orc, "baryon_mass", wrong_lambda)
    R1, R2 = _normalised_pair(L, ids, m_ud, m_s, 2, 7)
    assert all(np.abs(R1[i] - R2[i]).max() > 1e-6 * np.abs(R1[i]).max() for i in range(3))

    monkeypatch.setattr(orc, "baryon_mass", lambda name, a, b: -good(name, a, b))
    R1, R2 = _normalised_pair(L, ids, m_ud, m_s, 2, 7)
    assert all(np.abs(R1[i] - R2[i]).max() > 1e-6 * np.abs(R1[i]).max() for i in range(4))
