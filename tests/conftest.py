import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import wholeevents  # noqa: E402


def pytest_configure(config):
    # temporary files of the tests stay inside the repository, whatever the
    # working directory
    if not config.option.basetemp:
        config.option.basetemp = os.path.join(ROOT, ".pytest_tmp")
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


def pytest_collection_finish(session):
    # the oracle's whole-event results take minutes: start them in
    # background processes as soon as the tests that need them are selected
    if session.config.option.collectonly:
        return
    if any(item.nodeid.split("::")[0].endswith(wholeevents.TEST_FILE) for item in session.items):
        wholeevents.start()


def pytest_sessionfinish(session, exitstatus):
    wholeevents.stop()
