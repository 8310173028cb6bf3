"""GPU energy-to-solution from NVML's total-energy counter (read-only).

Energy-to-solution (Sec. 4, Table 3) is the energy a run draws; here it is
the difference of the device's cumulative energy counter (millijoules since
the GPU's kernel module loaded) around the run, for the GPU that runs it.  Only NVML's
query calls are made: nothing is set, locked or reset.  The library is
loaded through ctypes (no Python NVML package is needed); a missing
library, an unsupported counter or any NVML error leaves the meter
unavailable and its readings None.
"""
import ctypes
import os


class _Nvml:
    """The four NVML entry points used, over a loaded libnvidia-ml."""

    def __init__(self, lib):
        self.lib = lib

    def init(self):
        return self.lib.nvmlInit_v2()

    def handle_by_pci(self, bus_id):
        h = ctypes.c_void_p()
        rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus_id.encode()), ctypes.byref(h))
        return rc, h

    def handle_by_index(self, index):
        h = ctypes.c_void_p()
        rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h))
        return rc, h

    def total_energy_mj(self, h):
        e = ctypes.c_ulonglong()
        rc = self.lib.nvmlDeviceGetTotalEnergyConsumption(h, ctypes.byref(e))
        return rc, e.value

    def shutdown(self):
        return self.lib.nvmlShutdown()


def _load_nvml():
    for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
        try:
            return _Nvml(ctypes.CDLL(name))
        except OSError:
            continue
    return None


def _cuda_pci_bus_id(device):
    try:
        import torch
        p = torch.cuda.get_device_properties(device)
        return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    except Exception:
        return None


class EnergyMeter:
    """Cumulative GPU energy of one CUDA device.

    ``start()`` and ``stop()`` bracket a run (after a device synchronisation
    on both sides); ``joules`` is the energy between them, or None when the
    counter is unavailable.  ``nvml`` may be given (an object with the
    methods of ``_Nvml``) instead of loading the library; ``bus_id`` picks
    the device by PCI address, else the CUDA device's own address, else
    NVML index ``index``.
    """

    def __init__(self, device=0, nvml=None, bus_id=None, index=None):
        self.reason = None
        self._h = None
        self._nvml = nvml if nvml is not None else _load_nvml()
        self._e0 = self._e1 = None
        if self._nvml is None:
            self.reason = "NVML library not found"
            return
        if self._nvml.init() != 0:
            self.reason = "nvmlInit failed"
            self._nvml = None
            return
        bus = bus_id if bus_id is not None else (None if index is not None else _cuda_pci_bus_id(device))
        rc, h = self._nvml.handle_by_pci(bus) if bus else (1, None)
        if rc != 0:
            idx = index if index is not None else _visible_index(device)
            rc, h = self._nvml.handle_by_index(idx)
        if rc != 0:
            self.reason = "no NVML handle for the device"
            return
        rc, _ = self._nvml.total_energy_mj(h)
        if rc != 0:
            self.reason = "total energy counter not supported"
            return
        self._h = h

    @property
    def available(self):
        return self._h is not None

    def read_mj(self):
        """The device's cumulative energy in millijoules (None if unavailable)."""
        if self._h is None:
            return None
        rc, e = self._nvml.total_energy_mj(self._h)
        return e if rc == 0 else None

    def start(self):
        self._e0, self._e1 = self.read_mj(), None

    def stop(self):
        self._e1 = self.read_mj()
        return self.joules

    @property
    def joules(self):
        if self._e0 is None or self._e1 is None or self._e1 < self._e0:
            return None
        return (self._e1 - self._e0) / 1000.0

    def close(self):
        if self._nvml is not None:
            self._nvml.shutdown()
            self._nvml = None
            self._h = None


def _visible_index(device):
    """NVML index of CUDA device `device` when CUDA_VISIBLE_DEVICES lists plain indices."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p.strip() for p in vis.split(",") if p.strip()]
    if device < len(parts) and parts[device].isdigit():
        return int(parts[device])
    return int(device)
