"""Read-only SM clock sampling during a timed region.

Samples the SM clock and the clock-event (throttle) reasons of one GPU in a
background thread through NVML (``libnvidia-ml.so.1`` from the driver, via
ctypes) every ~2 ms, so even a short timed region gets samples.  If NVML
cannot be loaded it falls back to ``nvidia-smi -lms 50``.  Nothing here
changes any GPU setting.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading
import time

REASONS = {
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
    0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
    0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting",
}
NVML_CLOCK_SM = 1


class ClockSampler:
    def __init__(self, index: int = 0, period_s: float = 0.00025):
        self.index = index
        self.period = period_s
        self.samples = []          # (sm_mhz, reasons_mask)
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self._smi = None
        self._smi_file = None
        self._nvml = None
        self._handle = None
        self._init_nvml()

    def _init_nvml(self):
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                return
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self._nvml, self._handle = lib, h
        except OSError:
            self._nvml = None

    def _reasons_fn(self):
        for name in ("nvmlDeviceGetCurrentClocksEventReasons", "nvmlDeviceGetCurrentClocksThrottleReasons"):
            fn = getattr(self._nvml, name, None)
            if fn is not None:
                return fn
        return None

    def _run(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        rfn = self._reasons_fn()
        while not self._stop.is_set():
            if self._nvml.nvmlDeviceGetClockInfo(self._handle, NVML_CLOCK_SM, ctypes.byref(clk)) == 0:
                r = rs.value if (rfn is not None and rfn(self._handle, ctypes.byref(rs)) == 0) else 0
                self.samples.append((float(clk.value), int(r)))
            time.sleep(self.period)

    def start(self):
        self.samples = []
        self._stop.clear()
        if self._nvml is not None:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
            return
        try:
            fd, path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self._smi_file = path
            self._smi = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.active", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self._smi = None

    def stop(self) -> dict:
        if self._thread is not None:
            self._stop.set()
            self._thread.join()
            self._thread = None
        elif self._smi is not None:
            self._smi.terminate()
            self._smi.wait()
            for line in open(self._smi_file):
                parts = [p.strip() for p in line.split(",")]
                try:
                    self.max_mhz = float(parts[1])
                    self.samples.append((float(parts[0]), int(parts[2], 16)))
                except (ValueError, IndexError):
                    pass
            os.unlink(self._smi_file)
            self._smi = None
        return self.summary()

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0}
        mhz = sorted(s[0] for s in self.samples)
        mask = 0
        for _, r in self.samples:
            mask |= r
        reasons = [name for bit, name in sorted(REASONS.items()) if mask & bit and bit != 0x1]
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(self.samples), "source": "nvml" if self._nvml is not None else "nvidia-smi"}
