"""Seeded synthetic raw data shaped like a vacuum-fluctuation homodyne QRNG.

This module is the one place both the CUDA path (tests, benchmark) and the
CPU oracle take their inputs from.  It holds none of the extractor's
arithmetic: it draws Gaussian noise, quantises it like an ADC and describes
the benchmark workloads.  Packing samples into a bit stream is the
extractor's ingest step and is done by the oracle and by the GPU kernel,
each on its own.

Recipe (stand-in for the homodyne raw data of the paper's Sec. 4.2, which is
not available here):
  g ~ N(0, 1) from numpy ``Generator(PCG64(seed))``;
  v = sigma(t) * g + offset(t);
  sample = clamp(floor((v + 4) / 8 * 2^b), 0, 2^b - 1)   (ADC clipped at +-4)
Optional per-sample bias offset ~ U(-a, a) and slow sinusoidal drift of sigma.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def adc_samples(seed: int, nsamples: int, b: int, sigma: float = 1.0, offset_amp: float = 0.0,
                drift_amp: float = 0.0, drift_period: float | None = None,
                start: int = 0) -> np.ndarray:
    """Quantised Gaussian ADC samples (uint16 holding b-bit codes).

    ``start`` offsets the drift phase so a long stream can be generated in
    chunks; the noise itself comes from the seed alone."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(nsamples)
    if offset_amp:
        # offsets from their own stream so any prefix of a stream is reproducible alone
        g = g + np.random.Generator(np.random.PCG64([seed, 1])).uniform(-offset_amp, offset_amp, nsamples)
    if drift_amp:
        period = float(drift_period or nsamples)
        t = np.arange(start, start + nsamples, dtype=np.float64)
        g = g * (sigma * (1.0 + drift_amp * np.sin(2.0 * math.pi * t / period)))
    elif sigma != 1.0:
        g = g * sigma
    v = np.floor((g + 4.0) / 8.0 * float(1 << b))
    return np.clip(v, 0, (1 << b) - 1).astype(np.uint16)


def adc_samples_device(seed: int, nsamples: int, b: int, device, chunk: int = 1 << 25):
    """Quantised Gaussian ADC samples drawn on the device by torch's seeded
    generator, for workloads too large to draw on the host: N(0,1) noise
    clipped at +-4 sigma and quantised to b-bit codes, floor((g + 4)/8 * 2^b),
    as adc_samples does, with a different random source.  Returns an int16
    tensor holding the codes (uint16 bit patterns)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty(nsamples, dtype=torch.int16, device=device)
    scale = float(1 << b) / 8.0
    for a in range(0, nsamples, chunk):
        k = min(chunk, nsamples - a)
        g = torch.randn(k, generator=gen, device=device, dtype=torch.float32)
        v = torch.clamp(torch.floor((g + 4.0) * scale), 0, (1 << b) - 1)
        out[a:a + k] = v.to(torch.int32).to(torch.int16)
    return out


def random_words(seed: int, nwords: int) -> np.ndarray:
    """Uniformly random uint32 words (full-entropy test input)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 1 << 32, size=nwords, dtype=np.uint64).astype(np.uint32)


def _phi(x: float) -> float:
    return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))


def adc_min_entropy(b: int, sigma: float = 1.0, offset_amp: float = 0.0) -> float:
    """Classical min-entropy -log2 max_v P(sample = v) of the quantiser above,
    worst case over offsets in [-offset_amp, offset_amp] (a bin centred on the
    mean is the most likely outcome; the worst offset centres one)."""
    w = 8.0 / float(1 << b)
    centred = 2.0 * _phi(w / (2.0 * sigma)) - 1.0
    aligned = _phi(w / sigma) - 0.5
    p = centred if offset_amp >= w / 2.0 else aligned
    return -math.log2(p)


def block_min_entropy(n: int, b: int, h_sample: float) -> int:
    """Min-entropy credited to one n-bit block: whole samples only, minus the
    one a block boundary may split when b does not divide n."""
    whole = n // b - (1 if n % b else 0)
    return int(math.floor(h_sample * whole))


@dataclass
class StreamSpec:
    """One pair of raw streams for the extractor."""
    n: int                 # block length in bits (the paper's q*n)
    nblocks: int           # whole blocks per source
    b: int                 # ADC bits per sample
    seed_x: int
    seed_y: int
    eps: float             # per-block error target (Definition 2.3's epsilon)
    offset_amp: float = 0.0
    sigma: float = 1.0
    drift_amp: float = 0.0
    k: int = field(default=0)

    def __post_init__(self):
        if not self.k:
            s = self.sigma * (1.0 - self.drift_amp)
            self.k = block_min_entropy(self.n, self.b, adc_min_entropy(self.b, s, self.offset_amp))

    @property
    def nbits(self) -> int:
        return self.n * self.nblocks

    @property
    def nsamples(self) -> int:
        return -(-self.nbits // self.b)

    def samples(self, which: str) -> np.ndarray:
        seed = self.seed_x if which == "x" else self.seed_y
        return adc_samples(seed, self.nsamples, self.b, sigma=self.sigma, offset_amp=self.offset_amp,
                           drift_amp=self.drift_amp, drift_period=self.nsamples if self.drift_amp else None)


# Per-block eps targets: the paper's whole-stream 2^-30 (Sec. 4.2) split over
# the blocks of a stream by Theorem 3.3's sum; 256-bit blocks cannot reach
# that and use 2^-9 per block (a parity / latency workload).
EPS_BLOCK = {256: 2.0 ** -9, 1024: 2.0 ** -50, 4096: 2.0 ** -52}
# Mixed 8/12-bit workloads: 1024-bit blocks of 8-bit samples carry k = 809,
# whose q = 16 bound is 2^-41.7 per block; 2^-40 keeps q = n/64 for both b.
EPS_BLOCK_MIXED = {256: 2.0 ** -9, 1024: 2.0 ** -40, 4096: 2.0 ** -52}


def config_plain_small() -> StreamSpec:
    """4096 blocks x 256 bits per source, 8-bit ADC, seeds 0 / 1."""
    return StreamSpec(n=256, nblocks=4096, b=8, seed_x=0, seed_y=1, eps=EPS_BLOCK[256])


def config_large_single(nblocks: int = 1 << 20) -> StreamSpec:
    """2^20 blocks x 1024 bits per source (1 Gbit each), 12-bit ADC with a
    per-sample bias offset U(-0.05, 0.05) sigma."""
    return StreamSpec(n=1024, nblocks=nblocks, b=12, seed_x=0, seed_y=1, eps=EPS_BLOCK[1024],
                      offset_amp=0.05)


def config_batched(master_seed: int = 3, nstreams: int = 64, lo: int = 12, hi: int = 20):
    """64 stream pairs, block counts 2^U with U ~ U(lo, hi) rounded, n over
    {256, 1024, 4096}, b over {8, 12}; stream s uses seeds 2s, 2s+1."""
    rng = np.random.Generator(np.random.PCG64(master_seed))
    specs = []
    for s in range(nstreams):
        u = int(round(rng.uniform(lo, hi)))
        n = int(rng.choice([256, 1024, 4096]))
        b = int(rng.choice([8, 12]))
        specs.append(StreamSpec(n=n, nblocks=1 << u, b=b, seed_x=2 * s, seed_y=2 * s + 1, eps=EPS_BLOCK_MIXED[n]))
    return specs


def config_sustained(total_bits: int = 1 << 34, chunk_bits: int = 1 << 31) -> StreamSpec:
    """Two long 12-bit streams, n = 4096, sigma drifting +-5% sinusoidally over
    the stream; fed in chunks of ``chunk_bits`` (256 MiB = 2^31 bits)."""
    return StreamSpec(n=4096, nblocks=total_bits // 4096, b=12, seed_x=10, seed_y=11, eps=EPS_BLOCK[4096],
                      drift_amp=0.05)


def serving_requests(seed: int = 4, nreq: int = 256, nchannels: int = 256, rate: float = 2000.0,
                     lo: int = 10, hi: int = 18):
    """Poisson arrivals (exponential gaps at ``rate`` per second) from
    ``nchannels`` channels; each request carries 2^U block pairs, U ~ U(lo, hi),
    n over {256, 1024, 4096}, 12-bit ADC.  A channel keeps one n."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chan_n = rng.choice([256, 1024, 4096], size=nchannels)
    t = 0.0
    out = []
    for r in range(nreq):
        t += float(rng.exponential(1.0 / rate))
        c = int(rng.integers(0, nchannels))
        u = int(round(rng.uniform(lo, hi)))
        out.append(dict(id=r, t=t, channel=c, n=int(chan_n[c]), nblocks=1 << u, b=12,
                        seed_x=1000 + 2 * r, seed_y=1001 + 2 * r))
    return out
