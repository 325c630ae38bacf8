"""Seeded synthetic uplink subframes (the only code the oracle and the CUDA path share).

This module draws inputs; it holds none of the receiver's arithmetic (no LS, no
correlation model, no LMMSE weights, no detection, no demapping).  What it does:

* a multipath channel per (antenna, user): ``n_taps`` Rayleigh taps at integer
  delays 0..n_taps-1 with an exponential power-delay profile p_l ~ exp(-l/tau_rms)
  normalised to unit total power (Sec. III-A model under Eq. 16, Table III uses
  integer delays too), taken to the frequency domain over ``n_fft`` bins (Eq. 1-5);
* unit-modulus pilots with seeded phases, one pilot observation per user and slot
  (idealised orthogonal pilots: y_p = H p + n, Eq. 5 with one active user), or the comb
  of Sec. II (user k on tones k, k + S, ...; ``make_comb_subframe``);
* uniform payload labels mapped to Gray QAM (transmitter side): per dimension
  m = q/2 bits, read MSB first, even-indexed label bits on I and odd-indexed on Q,
  level = (2^m - 1) - 2 * gray_to_binary(bits), scaled to unit mean energy;
* data observations y = H x + n per subcarrier (Eq. 7) and AWGN of variance
  sigma2 = 10^(-SNR/10).

Everything is complex128; ``as_c64`` rounds what a receiver consumes to complex64
so both sides read bit-identical inputs.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_BASE = 0x18020542


@dataclasses.dataclass
class SubframeShape:
    M: int            # base-station antennas
    K: int            # single-antenna users
    n_sc: int         # used subcarriers
    n_fft: int        # FFT size (sets the tap phase step)
    n_taps: int = 6   # channel taps at delays 0..n_taps-1
    tau_rms: float = 4.0
    snr_db: float = 10.0
    qam_bits: int = 2
    n_slots: int = 2          # one pilot OFDM symbol per slot
    n_data_per_slot: int = 6  # data OFDM symbols per slot

    @property
    def sigma2(self) -> float:
        return float(10.0 ** (-self.snr_db / 10.0))

    @property
    def n_data(self) -> int:
        return self.n_slots * self.n_data_per_slot


def _cn(rng: np.random.Generator, shape, var) -> np.ndarray:
    """Circularly-symmetric complex Gaussian samples of variance ``var``."""
    s = np.sqrt(np.asarray(var, dtype=np.float64) / 2.0)
    return s * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def pdp_exponential(n_taps: int, tau_rms: float) -> np.ndarray:
    """Tap powers p_l = exp(-l/tau_rms) / sum, l = 0..n_taps-1 (generator's channel law)."""
    l = np.arange(n_taps, dtype=np.float64)
    p = np.exp(-l / tau_rms)
    return p / p.sum()


def gray_qam_map(labels: np.ndarray, qam_bits: int) -> np.ndarray:
    """Transmitter Gray-QAM mapper: integer labels (b0 = MSB) -> unit-energy symbols."""
    q = qam_bits
    m = q // 2
    labels = np.asarray(labels, dtype=np.int64)

    def pam(bit_positions):
        g = np.zeros(labels.shape, dtype=np.int64)
        for pos in bit_positions:          # MSB first
            g = (g << 1) | ((labels >> (q - 1 - pos)) & 1)
        u = g.copy()                      # gray -> binary: u = g ^ (g>>1) ^ (g>>2) ...
        shift = g >> 1
        while np.any(shift):
            u ^= shift
            shift >>= 1
        return ((1 << m) - 1) - 2 * u

    i_lvl = pam(range(0, q, 2))
    q_lvl = pam(range(1, q, 2))
    scale = np.sqrt(2.0 * (4 ** m - 1) / 3.0)
    return (i_lvl + 1j * q_lvl) / scale


def make_subframe(shape: SubframeShape, seed: int, noiseless: bool = False,
                  pilot_modulus: Optional[np.ndarray] = None) -> dict:
    """Draw one subframe.

    Returns a dict of complex128 / int arrays:
      H        [M][K][n_sc]                true channel per subcarrier
      pilots   [n_slots][K][n_sc]          unit-modulus pilots (or scaled by pilot_modulus)
      y_pilot  [n_slots][K][M][n_sc]       per-user pilot observation
      labels   [n_data][K][n_sc]           transmitted Gray labels (int)
      x        [n_data][K][n_sc]           transmitted symbols
      y_data   [n_data][M][n_sc]           received data symbols
      sigma2   float                       noise variance used (0 if noiseless)
    """
    sh = shape
    rng = np.random.default_rng(seed)
    p_l = pdp_exponential(sh.n_taps, sh.tau_rms)
    taps = _cn(rng, (sh.M, sh.K, sh.n_taps), p_l[None, None, :])
    k = np.arange(sh.n_sc, dtype=np.float64)
    l = np.arange(sh.n_taps, dtype=np.float64)
    steer = np.exp(-2j * np.pi * np.outer(l, k) / sh.n_fft)      # [n_taps][n_sc]
    H = taps @ steer                                               # [M][K][n_sc]

    theta = rng.uniform(0.0, 2.0 * np.pi, size=(sh.n_slots, sh.K, sh.n_sc))
    pilots = np.exp(1j * theta)
    if pilot_modulus is not None:
        pilots = pilots * pilot_modulus

    sigma2 = 0.0 if noiseless else sh.sigma2
    Ht = np.transpose(H, (1, 0, 2))                                # [K][M][n_sc]
    n_p = _cn(rng, (sh.n_slots, sh.K, sh.M, sh.n_sc), sigma2)
    y_pilot = Ht[None, :, :, :] * pilots[:, :, None, :] + n_p

    labels = rng.integers(0, 1 << sh.qam_bits, size=(sh.n_data, sh.K, sh.n_sc))
    x = gray_qam_map(labels, sh.qam_bits)
    n_d = _cn(rng, (sh.n_data, sh.M, sh.n_sc), sigma2)
    y_data = np.einsum("mkn,dkn->dmn", H, x) + n_d
    return dict(H=H, pilots=pilots, y_pilot=y_pilot, labels=labels, x=x,
                y_data=y_data, sigma2=sigma2, taps=taps, pdp=p_l)


def make_comb_subframe(shape: SubframeShape, seed: int, S: int, noiseless: bool = False,
                       tap_powers: Optional[np.ndarray] = None) -> dict:
    """Draw one subframe with the comb pilot structure of Sec. II (Fig. 1).

    The pilot OFDM symbol of each slot is shared: user k owns the tones n with n mod S == k
    (tones of offsets >= K carry no user, only noise).  ``tap_powers`` (optional) replaces
    the exponential profile with given tap powers at delays 0, 1, ... (normalised).

    Returns, besides H, labels, x, y_data and sigma2 as in make_subframe:
      pilots   [n_slots][n_sc]       unit-modulus value sent on each tone by its owner
      y_pilot  [n_slots][M][n_sc]    received pilot symbol
    """
    sh = shape
    if sh.K > S:
        raise ValueError("K users need at least K comb offsets")
    rng = np.random.default_rng(seed)
    if tap_powers is None:
        p_l = pdp_exponential(sh.n_taps, sh.tau_rms)
    else:
        p_l = np.asarray(tap_powers, dtype=np.float64)
        p_l = p_l / p_l.sum()
    n_taps = p_l.size
    taps = _cn(rng, (sh.M, sh.K, n_taps), p_l[None, None, :])
    k = np.arange(sh.n_sc, dtype=np.float64)
    l = np.arange(n_taps, dtype=np.float64)
    H = taps @ np.exp(-2j * np.pi * np.outer(l, k) / sh.n_fft)    # [M][K][n_sc]

    pilots = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=(sh.n_slots, sh.n_sc)))
    owner = np.arange(sh.n_sc) % S
    sigma2 = 0.0 if noiseless else sh.sigma2
    Hown = np.zeros((sh.M, sh.n_sc), dtype=np.complex128)
    live = owner < sh.K
    Hown[:, live] = H[:, owner[live], np.arange(sh.n_sc)[live]]
    y_pilot = Hown[None] * pilots[:, None, :] + _cn(rng, (sh.n_slots, sh.M, sh.n_sc), sigma2)

    labels = rng.integers(0, 1 << sh.qam_bits, size=(sh.n_data, sh.K, sh.n_sc))
    x = gray_qam_map(labels, sh.qam_bits)
    y_data = np.einsum("mkn,dkn->dmn", H, x) + _cn(rng, (sh.n_data, sh.M, sh.n_sc), sigma2)
    return dict(H=H, pilots=pilots, y_pilot=y_pilot, labels=labels, x=x,
                y_data=y_data, sigma2=sigma2, taps=taps, pdp=p_l)


def as_c64(a: np.ndarray) -> np.ndarray:
    """Round to the complex64 values a receiver reads (contiguous)."""
    return np.ascontiguousarray(np.asarray(a).astype(np.complex64))


# Workloads named by what they are (M x K, subcarriers, FFT, modulation, PDP).
TINY = SubframeShape(M=8, K=2, n_sc=72, n_fft=128, n_taps=6, tau_rms=4.0,
                     snr_db=10.0, qam_bits=2)
PAPER_SCALE = SubframeShape(M=128, K=12, n_sc=1200, n_fft=2048, n_taps=24,
                            tau_rms=8.0, snr_db=10.0, qam_bits=4)
