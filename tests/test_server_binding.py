"""Host logic of the Server binding (no GPU): Server.forget maps the library's status to
IgpError and releases the binding's reference to an output only when the library dropped the
request. The library is replaced by a fake with the same call signatures."""
import ctypes

import numpy as np
import pytest

from paper_2508_19737_gb300 import api


class _FakeLib:
    def __init__(self):
        self.next_ticket = 1
        self.state = {}  # ticket -> "queued" | "done"
        self.err = b""

    def igp_embed_opts_init(self, o):
        pass

    def igp_server_opts_init(self, o):
        pass

    def igp_server_create(self, o, h):
        h._obj.value = 1234
        return api.IGP_OK

    def igp_submit(self, handle, r, t):
        t._obj.value = self.next_ticket
        self.state[self.next_ticket] = "queued"
        self.next_ticket += 1
        return api.IGP_OK

    def igp_server_forget(self, handle, ticket):
        if ticket not in self.state:
            self.err = b"unknown ticket"
            return api.IGP_E_INVAL
        if self.state[ticket] != "done":
            self.err = b"queued"
            return api.IGP_E_BUSY
        del self.state[ticket]
        return api.IGP_OK

    def igp_last_error(self):
        return self.err

    def igp_server_destroy(self, handle):
        pass


def test_forget_releases_the_output_only_once_dropped(monkeypatch):
    fake = _FakeLib()
    monkeypatch.setattr(api, "lib", lambda: fake)
    sv = api.Server(slots=1)
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    t = sv.submit(src, dst, 3, -0.5, 2, 8, 0)
    out = sv.result(t)
    assert out.shape == (3, 8) and out.dtype == np.float32
    with pytest.raises(api.IgpError) as e:  # still queued: nothing is released
        sv.forget(t)
    assert e.value.status == api.IGP_E_BUSY
    assert sv.result(t) is out
    fake.state[t] = "done"
    assert sv.forget(t) is out
    with pytest.raises(KeyError):
        sv.result(t)
    with pytest.raises(api.IgpError) as e:
        sv.forget(t)
    assert e.value.status == api.IGP_E_INVAL
    sv.close()
    assert sv.handle is None
