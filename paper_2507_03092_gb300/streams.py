"""Seeded outcome-coin and noise-draw streams (input generator).

Every random choice the simulation makes is an *input*: random measurement
outcomes read a coin bit, noise channels read a 32-bit draw.  Both come from
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), a counter-based generator: output k of a stream
with key s is mix64(s + (k+1)*GAMMA).

Stream layout (per shot):
  coins: uint64 words; coin for the m-th M/R op (circuit order) is bit m%64 of
         word m//64.  Word k = splitmix64(key(seed, shot, COIN), k).
  noise: uint32 words; the l-th noise op reads word l (RESET_ERROR reads three
         consecutive words).  Word l = splitmix64(key(seed, shot, NOISE), l) >> 32.
  key(seed, shot, kind) = mix64(mix64(seed + kind*GAMMA) + (shot+1)*GAMMA).

This module holds no simulation arithmetic; the GPU's on-the-fly stream mode
implements the same published generator independently.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
KIND_COIN = 1
KIND_NOISE = 2
_M64 = (1 << 64) - 1


def mix64_int(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * MIX1) & _M64
    z = ((z ^ (z >> 27)) * MIX2) & _M64
    return z ^ (z >> 31)


def stream_key(seed: int, shot: int, kind: int) -> int:
    return mix64_int((mix64_int((seed + kind * GAMMA) & _M64) + (shot + 1) * GAMMA) & _M64)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(MIX1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(MIX2)
        z ^= z >> np.uint64(31)
    return z


def splitmix64(key: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 stream with state ``key``."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + k * np.uint64(GAMMA)
    return _mix64_np(z)


def coin_words(seed: int, shots, n_words: int) -> np.ndarray:
    """uint64 [len(shots), n_words]."""
    shots = np.atleast_1d(np.asarray(shots, dtype=np.int64))
    out = np.empty((len(shots), max(1, n_words)), dtype=np.uint64)
    for i, s in enumerate(shots):
        out[i] = splitmix64(stream_key(seed, int(s), KIND_COIN), out.shape[1])
    return out


def noise_words(seed: int, shots, n_words: int) -> np.ndarray:
    """uint32 [len(shots), n_words]."""
    shots = np.atleast_1d(np.asarray(shots, dtype=np.int64))
    out = np.empty((len(shots), max(1, n_words)), dtype=np.uint32)
    for i, s in enumerate(shots):
        out[i] = (splitmix64(stream_key(seed, int(s), KIND_NOISE), out.shape[1])
                  >> np.uint64(32)).astype(np.uint32)
    return out


def streams_for(circuit, seed: int, shots) -> tuple[np.ndarray, np.ndarray]:
    """(coins uint64 [S, coin_words], noise uint32 [S, noise_words]) for ``circuit``."""
    return (coin_words(seed, shots, circuit.coin_words),
            noise_words(seed, shots, circuit.noise_words))


def shot_distances(seed: int, shots: int, choices=(3, 5, 7, 9, 11)) -> np.ndarray:
    """Per-shot code distance for the mixed-distance batch: choices[
    splitmix64(key(seed, shot, 3), 0) mod len(choices)]."""
    out = np.empty(shots, dtype=np.int64)
    for s in range(shots):
        v = int(splitmix64(stream_key(seed, s, 3), 1)[0])
        out[s] = choices[v % len(choices)]
    return out
