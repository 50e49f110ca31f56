"""Mlp.save / load_mlp, the learned functional's checkpoint file, on the CPU:
the file holds the state, step and box the network reports, and loading
creates a network from the parameters and box and restores the whole state
(the network itself is stood in for; its state round trip on the GPU is
test_gpu_mlp.py::test_checkpoint_resumes_training_bit_for_bit)."""
import numpy as np
import pytest


def _kldi():
    from paper_2605_10363_gb300 import kldi
    return kldi


class _Net:
    box = np.array([-30.0, 5.0, -69.0, 20.0])

    def state(self):
        kldi = _kldi()
        return np.linspace(-1.0, 1.0, 3 * kldi.MLP_NPARAMS, dtype=np.float32), 1234


def test_checkpoint_file_round_trip(tmp_path, monkeypatch):
    kldi = _kldi()
    path = str(tmp_path / "mlp.npz")
    kldi.Mlp.save(_Net(), path)
    with np.load(path) as z:
        assert sorted(z.files) == ["box", "state", "step"]
        assert z["state"].dtype == np.float32 and int(z["step"]) == 1234
    made = {}

    class Recorder:
        def __init__(self, params, box):
            made["params"], made["box"] = np.array(params), np.array(box)

        def set_state(self, state, step):
            made["state"], made["step"] = np.array(state), step

    monkeypatch.setattr(kldi, "Mlp", Recorder)
    kldi.load_mlp(path)
    state, step = _Net().state()
    assert np.array_equal(made["params"], state[:kldi.MLP_NPARAMS])
    assert np.array_equal(made["box"], _Net.box)
    assert np.array_equal(made["state"], state) and made["step"] == step


def test_malformed_checkpoints_are_refused(tmp_path):
    kldi = _kldi()
    good_state, _ = _Net().state()
    cases = {
        "short": dict(state=good_state[:10], step=np.int64(1), box=_Net.box),
        "box": dict(state=good_state, step=np.int64(1), box=_Net.box[:3]),
        "step": dict(state=good_state, step=np.int64(-1), box=_Net.box),
        "extra": dict(state=good_state, step=np.int64(1), box=_Net.box, other=np.zeros(1)),
    }
    for name, arrays in cases.items():
        path = str(tmp_path / f"{name}.npz")
        np.savez(path, **arrays)
        with pytest.raises(ValueError):
            kldi.load_mlp(path)
