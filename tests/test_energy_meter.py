"""Host logic of the NVML energy meter against a fake NVML (no GPU, no driver).

The fake records every call: the meter may only initialise, look up a handle,
read the total-energy counter and shut down.
"""
from paper_2608_24348_gb300.energy import EnergyMeter, _visible_index


class FakeNvml:
    def __init__(self, counter=(1000, 1500, 4250), init_rc=0, pci_rc=0, energy_rc=0):
        self.calls = []
        self.counter = list(counter)
        self.init_rc, self.pci_rc, self.energy_rc = init_rc, pci_rc, energy_rc

    def init(self):
        self.calls.append("init")
        return self.init_rc

    def handle_by_pci(self, bus_id):
        self.calls.append(("pci", bus_id))
        return self.pci_rc, "h-pci"

    def handle_by_index(self, index):
        self.calls.append(("index", index))
        return 0, f"h-{index}"

    def total_energy_mj(self, h):
        self.calls.append(("energy", h))
        if self.energy_rc:
            return self.energy_rc, 0
        return 0, self.counter.pop(0) if len(self.counter) > 1 else self.counter[0]

    def shutdown(self):
        self.calls.append("shutdown")
        return 0


def test_joules_between_start_and_stop():
    f = FakeNvml(counter=(1000, 1500, 4250))
    m = EnergyMeter(nvml=f, bus_id="00000000:1b:00.0")
    assert m.available
    m.start()
    assert m.stop() == (4250 - 1500) / 1000.0
    m.close()
    names = {c if isinstance(c, str) else c[0] for c in f.calls}
    assert names <= {"init", "pci", "index", "energy", "shutdown"}
    assert ("pci", "00000000:1b:00.0") in f.calls and f.calls[-1] == "shutdown"


def test_falls_back_to_the_index_when_the_bus_id_lookup_fails():
    f = FakeNvml(pci_rc=13)
    m = EnergyMeter(nvml=f, bus_id="00000000:1b:00.0", index=3)
    assert m.available and ("index", 3) in f.calls


def test_unavailable_counter_gives_none():
    for kw, why in ((dict(init_rc=9), "nvmlInit"), (dict(energy_rc=3), "not supported")):
        m = EnergyMeter(nvml=FakeNvml(**kw), bus_id="x")
        assert not m.available and why in m.reason
        m.start()
        assert m.stop() is None and m.read_mj() is None


def test_counter_that_went_backwards_gives_none():
    m = EnergyMeter(nvml=FakeNvml(counter=(10, 500, 100)), bus_id="x")
    m.start()
    assert m.stop() is None


def test_visible_index(monkeypatch):
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,2")
    assert _visible_index(1) == 2
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-abc")
    assert _visible_index(0) == 0
