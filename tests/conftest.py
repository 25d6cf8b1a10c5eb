import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_sessionfinish(session, exitstatus):
    """With the checking build loaded (OMERF_CHECK=1), no feature read of any
    scene the session created may have fallen outside its arrays."""
    if os.environ.get("OMERF_CHECK") != "1" or exitstatus != 0:
        return
    import gc
    gc.collect()
    try:
        import paper_2404_09531_gb300 as om
        if not om.lib().omerf_check_build():
            return
        unstored, outside = om.check_totals()
    except Exception:
        return
    print(f"\nchecking build: {outside} feature reads outside the arrays, {unstored} corner reads of unstored "
          f"bricks, over the session's scenes")
    if outside:
        session.exitstatus = 1
