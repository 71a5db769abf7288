"""Host-side fault injection (CPU): gs_debug_inject_failure arms one failure
of a call kind and refuses bad arguments; nothing here reaches a device."""
import pytest


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300

    return paper_2501_09398_gb300


def test_arm_and_disarm(g):
    g.gs_debug_inject_failure(g.GS_INJECT_NONE)
    assert not g.gs_debug_injection_pending()
    g.gs_debug_inject_failure(g.GS_INJECT_MALLOC, 3)
    assert g.gs_debug_injection_pending()
    g.gs_debug_inject_failure(g.GS_INJECT_GRAPH_NODE, 0)  # re-arming replaces the kind
    assert g.gs_debug_injection_pending()
    g.gs_debug_inject_failure(g.GS_INJECT_NONE)
    assert not g.gs_debug_injection_pending()


@pytest.mark.parametrize("call,after", [(3, 0), (-1, 0), (1, -1)])
def test_bad_arguments(g, call, after):
    with pytest.raises(g.GsError) as e:
        g.gs_debug_inject_failure(call, after)
    assert e.value.status == g.GS_ERR_INVALID_ARG
    assert not g.gs_debug_injection_pending()


def test_pending_needs_an_output(g):
    assert g.raw_call("gs_debug_injection_pending", None) == g.GS_ERR_INVALID_ARG
